/*
 * CPU oracle for the fixed-radius pair sum (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  It shares no code with the CUDA path.  Build with
 *   gcc -O2 -fPIC -shared -ffp-contract=off -fno-fast-math -fopenmp
 * so that every FP32 operation below is one correctly rounded IEEE-754
 * binary32 operation: -ffp-contract=off forbids FMA contraction, and on the
 * x86-64 (SSE) and AArch64 targets float arithmetic carries no excess
 * precision (FLT_EVAL_METHOD == 0, checked at compile time below).
 *
 * What it computes (paper Sec. 1 problem statement, Sec. 2.2.1-2.2.2 and
 * Sec. 3, Eq. 1 and the velocity-update listing):
 *   N particles in a d-dimensional box [lo, hi), each axis periodic or not;
 *   the neighbours of i are all j != i whose shortest (minimum-image)
 *   separation dx_ij = r_j - r_i has |dx_ij| < r;
 *   y_i = sum over neighbours of f(dx_ij, v_i, v_j).
 *
 * Readings of the paper used here (the paper only says "shortest vector"):
 *   1. minimum image per periodic axis k, in FP32 round-to-nearest:
 *        dx = x_j - x_i;  if dx > halfL: dx = dx - L;
 *                         else if dx < -halfL: dx = dx + L;
 *      with L = hi - lo and halfL = 0.5f * L, both rounded to FP32;
 *   2. d2 = (dx0*dx0 + dx1*dx1) + dx2*dx2 evaluated left to right in FP32;
 *   3. (i, j) is a pair iff j != i and d2 < r2, r2 = (float)r * (float)r
 *      rounded once to FP32 (strict "<" as in Eq. 1).
 *   Values are then evaluated in FP64 from the FP32 positions, re-using the
 *   wrap decision taken in FP32 so that the image is the same one.
 *
 * Two independent neighbour searches:
 *   - or_brute_*: the definition itself, O(N) per query, no cells;
 *   - or_cells_*: a textbook linked-list cell list (head/next) whose cell
 *     index is computed in FP64 with width >= r(1+1e-5) + 1e-6 L, so that the
 *     3^d stencil covers every pair the FP32 predicate can accept.
 * Rows of every CSR result are sorted by ascending j.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs float arithmetic evaluated in float"
#endif

/* ------------------------------------------------------------------------ */
/* Box description shared by all entry points.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dim;
    int periodic[3];
    float lo[3];
    float hi[3];
    float L[3];      /* hi - lo in FP32 */
    float halfL[3];  /* 0.5f * L in FP32 */
    float r2;        /* r*r in FP32 */
} box_t;

static void box_init(box_t *b, int dim, const int *periodic, const float *lo,
                     const float *hi, float r) {
    memset(b, 0, sizeof(*b));
    b->dim = dim;
    for (int k = 0; k < dim; ++k) {
        float l = hi[k] - lo[k];
        float h = 0.5f * l;
        b->periodic[k] = periodic[k] ? 1 : 0;
        b->lo[k] = lo[k];
        b->hi[k] = hi[k];
        b->L[k] = l;
        b->halfL[k] = h;
    }
    float rr = r * r;
    b->r2 = rr;
}

/* Reading 1: FP32 minimum image of x_j - x_i along one axis; *wrap receives
 * the multiple of L that was added (-1, 0 or +1). */
static float min_image_f32(const box_t *b, int k, float xi, float xj, int *wrap) {
    float dx = xj - xi;
    *wrap = 0;
    if (b->periodic[k]) {
        if (dx > b->halfL[k]) {
            dx = dx - b->L[k];
            *wrap = -1;
        } else if (dx < -b->halfL[k]) {
            dx = dx + b->L[k];
            *wrap = +1;
        }
    }
    return dx;
}

/* Readings 2 and 3: FP32 squared distance in fixed order, strict test. */
static int is_pair(const box_t *b, const float *pi, const float *pj) {
    int w;
    float d0 = min_image_f32(b, 0, pi[0], pj[0], &w);
    float d1 = min_image_f32(b, 1, pi[1], pj[1], &w);
    float s0 = d0 * d0;
    float s1 = d1 * d1;
    float d2 = s0 + s1;
    if (b->dim == 3) {
        float d2z = min_image_f32(b, 2, pi[2], pj[2], &w);
        float s2 = d2z * d2z;
        d2 = d2 + s2;
    }
    return d2 < b->r2;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------ */
/* Brute force (the plain definition).                                      */
/* pos: float32[n][4]; queries: int64[nq]; counts: int64[nq].              */
/* ------------------------------------------------------------------------ */
void or_brute_counts(int dim, const int *periodic, const float *lo,
                     const float *hi, float r, int64_t n, const float *pos,
                     int64_t nq, const int64_t *queries, int64_t *counts) {
    box_t b;
    box_init(&b, dim, periodic, lo, hi, r);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = queries[q];
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i && is_pair(&b, pos + 4 * i, pos + 4 * j)) ++c;
        counts[q] = c;
    }
}

void or_brute_list(int dim, const int *periodic, const float *lo,
                   const float *hi, float r, int64_t n, const float *pos,
                   int64_t nq, const int64_t *queries, const int64_t *offsets,
                   int32_t *idx) {
    box_t b;
    box_init(&b, dim, periodic, lo, hi, r);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = queries[q];
        int64_t o = offsets[q];
        for (int64_t j = 0; j < n; ++j)
            if (j != i && is_pair(&b, pos + 4 * i, pos + 4 * j)) idx[o++] = (int32_t)j;
    }
}

/* ------------------------------------------------------------------------ */
/* Linked-list cell list with an FP64 cell index.                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    box_t b;
    int64_t n;
    const float *pos;   /* borrowed, float32[n][4] */
    int ncell[3];
    double width[3];
    int64_t total;
    int64_t *head;      /* [total], -1 terminated chains */
    int64_t *next;      /* [n] */
} or_cells;

static int cell_coord(const or_cells *cl, int k, float x) {
    double u = ((double)x - (double)cl->b.lo[k]) / cl->width[k];
    double f = floor(u);
    if (f < 0) f = 0;
    if (f > cl->ncell[k] - 1) f = cl->ncell[k] - 1;
    return (int)f;
}

or_cells *or_cells_build(int dim, const int *periodic, const float *lo,
                         const float *hi, float r, int64_t n, const float *pos) {
    or_cells *cl = (or_cells *)calloc(1, sizeof(or_cells));
    if (!cl) return NULL;
    box_init(&cl->b, dim, periodic, lo, hi, r);
    cl->n = n;
    cl->pos = pos;
    cl->total = 1;
    for (int k = 0; k < 3; ++k) {
        cl->ncell[k] = 1;
        cl->width[k] = 1.0;
    }
    for (int k = 0; k < dim; ++k) {
        double L = (double)hi[k] - (double)lo[k];
        double wmin = (double)r * (1.0 + 1e-5) + 1e-6 * L;
        double nc = floor(L / wmin);
        if (nc < 1) nc = 1;
        if (nc > 65536) nc = 65536;
        cl->ncell[k] = (int)nc;
    }
    /* Keep the head table modest: wider cells only add candidates. */
    for (;;) {
        int64_t t = 1;
        for (int k = 0; k < dim; ++k) t *= cl->ncell[k];
        if (t <= ((int64_t)1 << 26)) break;
        for (int k = 0; k < dim; ++k)
            cl->ncell[k] = cl->ncell[k] > 1 ? cl->ncell[k] / 2 : 1;
    }
    for (int k = 0; k < dim; ++k) {
        double L = (double)hi[k] - (double)lo[k];
        cl->width[k] = L / cl->ncell[k];
        cl->total *= (int64_t)cl->ncell[k];
    }
    cl->head = (int64_t *)malloc(sizeof(int64_t) * (size_t)cl->total);
    cl->next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cl->head || !cl->next) {
        free(cl->head);
        free(cl->next);
        free(cl);
        return NULL;
    }
    for (int64_t c = 0; c < cl->total; ++c) cl->head[c] = -1;
    /* Insert in descending index order so each chain is ascending in j. */
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t c = 0, stride = 1;
        for (int k = 0; k < dim; ++k) {
            c += stride * cell_coord(cl, k, pos[4 * i + k]);
            stride *= cl->ncell[k];
        }
        cl->next[i] = cl->head[c];
        cl->head[c] = i;
    }
    return cl;
}

void or_cells_free(or_cells *cl) {
    if (!cl) return;
    free(cl->head);
    free(cl->next);
    free(cl);
}

void or_cells_shape(const or_cells *cl, int *ncell) {
    for (int k = 0; k < 3; ++k) ncell[k] = cl->ncell[k];
}

/* Distinct neighbouring cell coordinates along axis k of cell c. */
static int axis_offsets(const or_cells *cl, int k, int c, int *out) {
    int n = cl->ncell[k], m = 0;
    if (k >= cl->b.dim) {
        out[0] = 0;
        return 1;
    }
    for (int o = -1; o <= 1; ++o) {
        int t = c + o;
        if (cl->b.periodic[k]) {
            t = ((t % n) + n) % n;
        } else if (t < 0 || t >= n) {
            continue;
        }
        int dup = 0;
        for (int u = 0; u < m; ++u) dup |= (out[u] == t);
        if (!dup) out[m++] = t;
    }
    return m;
}

/* Visit all candidates of query i; mode 0 counts, mode 1 writes. */
static int64_t cells_visit(const or_cells *cl, int64_t i, int32_t *dst) {
    const float *pi = cl->pos + 4 * i;
    int ci[3] = {0, 0, 0};
    for (int k = 0; k < cl->b.dim; ++k) ci[k] = cell_coord(cl, k, pi[k]);
    int ox[3], oy[3], oz[3];
    int nx = axis_offsets(cl, 0, ci[0], ox);
    int ny = axis_offsets(cl, 1, ci[1], oy);
    int nz = axis_offsets(cl, 2, ci[2], oz);
    int64_t cnt = 0;
    for (int a = 0; a < nz; ++a)
        for (int bq = 0; bq < ny; ++bq)
            for (int c = 0; c < nx; ++c) {
                int64_t cell = ox[c] + (int64_t)cl->ncell[0] *
                                           (oy[bq] + (int64_t)cl->ncell[1] * oz[a]);
                for (int64_t j = cl->head[cell]; j >= 0; j = cl->next[j]) {
                    if (j == i) continue;
                    if (is_pair(&cl->b, pi, cl->pos + 4 * j)) {
                        if (dst) dst[cnt] = (int32_t)j;
                        ++cnt;
                    }
                }
            }
    if (dst && cnt > 1) qsort(dst, (size_t)cnt, sizeof(int32_t), cmp_i32);
    return cnt;
}

void or_cells_counts(const or_cells *cl, int64_t nq, const int64_t *queries,
                     int64_t *counts) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t q = 0; q < nq; ++q) counts[q] = cells_visit(cl, queries[q], NULL);
}

void or_cells_list(const or_cells *cl, int64_t nq, const int64_t *queries,
                   const int64_t *offsets, int32_t *idx) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t q = 0; q < nq; ++q) cells_visit(cl, queries[q], idx + offsets[q]);
}

/* ------------------------------------------------------------------------ */
/* Pair operators in FP64 over a given neighbour CSR.                       */
/*                                                                          */
/* op 0 COUNT : y_i = #neighbours                                           */
/* op 1 GAUSS : y_i = sum_j w_j exp(-s d^2)                                 */
/* op 2 LJ    : y_i = 1/2 sum_j eps((sig/d)^12 - (sig/d)^6)   (truncated,   */
/*              unshifted; total energy = sum_i y_i)                        */
/* op 3 EXPF  : y_i = c sum_{j, d>0} -exp(-d) dx_ij / d      (Eq. 1)        */
/* op 4 SOFT  : y_i = sum_{j, d>0} -k (r - d) dx_ij / d                      */
/* op 5 SPH_DENSITY: rho_i = m_i W(0) + sum_j m_j W(d), w = m (float64[n]);  */
/*              Wendland C2 with support r: W(d) = a (1-q)^4 (1+4q), q=d/r, */
/*              a = 21/(2 pi r^3) (3-D), 7/(pi r^2) (2-D)                   */
/* op 6 SPH_FORCE: a_i = -sum_j m_j (A_i + A_j) grad_i W(d_ij),              */
/*              w = (m, A) per particle (float64[n][2], A = P/rho^2);       */
/*              grad_i W = W'(d) (x_i - x_j)/d, W'(d) = -20 a q (1-q)^3 / r  */
/*                                                                          */
/* pos64: float64[n][4]; w: float64[n] (GAUSS) or NULL; out: float64[nq][4] */
/* (scalar ops write out[q][0]).  prm = {s, eps, sigma, c, k, r}.           */
/* absmode != 0 sums |term| (componentwise; for LJ the two halves of the    */
/* potential, for SOFT the k r and k d parts, are added in magnitude) -- the */
/* denominator of the error metric.                                         */
/* ------------------------------------------------------------------------ */

/* FP64 separation with the image chosen by the FP32 rule. */
static double sep64(const box_t *b, int k, const double *pi, const double *pj) {
    int wrap;
    (void)min_image_f32(b, k, (float)pi[k], (float)pj[k], &wrap);
    return (pj[k] - pi[k]) + (double)wrap * (double)b->L[k];
}

void or_pair_eval(int op, int absmode, const double *prm, int dim,
                  const int *periodic,
                  const float *lo, const float *hi, int64_t n,
                  const double *pos64, const double *w, int64_t nq,
                  const int64_t *queries, const int64_t *offsets,
                  const int32_t *idx, double *out) {
    box_t b;
    box_init(&b, dim, periodic, lo, hi, (float)prm[5]);
    const double s = prm[0], eps = prm[1], sig = prm[2], c = prm[3],
                 kk = prm[4], r = prm[5];
    const double pi_ = 3.14159265358979323846;
    const double wend_a = dim == 3 ? 21.0 / (2.0 * pi_ * r * r * r) : 7.0 / (pi_ * r * r);
    (void)n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = queries[q];
        const double *pi = pos64 + 4 * i;
        double acc[4] = {0, 0, 0, 0};
        for (int64_t e = offsets[q]; e < offsets[q + 1]; ++e) {
            int64_t j = idx[e];
            const double *pj = pos64 + 4 * j;
            double dx[3] = {0, 0, 0}, d2 = 0;
            for (int k = 0; k < dim; ++k) {
                dx[k] = sep64(&b, k, pi, pj);
                d2 += dx[k] * dx[k];
            }
            double t[3] = {0, 0, 0};
            if (op == 0) {
                t[0] = 1.0;
            } else if (op == 1) {
                t[0] = w[j] * exp(-s * d2);
            } else if (op == 2) {
                double sr6 = pow(sig * sig / d2, 3);
                t[0] = absmode ? 0.5 * eps * (sr6 * sr6 + sr6)
                               : 0.5 * eps * (sr6 * sr6 - sr6);
            } else if (op == 3 || op == 4) {
                if (d2 > 0) {
                    double d = sqrt(d2);
                    double mag = (op == 3) ? -c * exp(-d) : -kk * (r - d);
                    /* k (r - d) cancels near the cut-off: the error metric
                     * counts the k r and k d parts in magnitude */
                    if (absmode && op == 4) mag = kk * (r + d);
                    for (int k = 0; k < dim; ++k) t[k] = mag * dx[k] / d;
                }
            } else if (op == 5) {
                const double q1 = sqrt(d2) / r, u = 1.0 - q1;
                t[0] = w[j] * wend_a * u * u * u * u * (1.0 + 4.0 * q1);
            } else if (op == 6) {
                /* a_i = sum_j m_j (A_i + A_j) W'(d)/d dx_ij, W'(d)/d = -20 a (1-q)^3 / r^2;
                 * the metric counts |A_i| + |A_j| */
                const double q1 = sqrt(d2) / r, u = 1.0 - q1;
                const double aa = absmode ? fabs(w[2 * i + 1]) + fabs(w[2 * j + 1])
                                          : w[2 * i + 1] + w[2 * j + 1];
                const double coef = w[2 * j] * aa * (-20.0 * wend_a * u * u * u / (r * r));
                for (int k = 0; k < dim; ++k) t[k] = coef * dx[k];
            }
            for (int k = 0; k < 3; ++k) acc[k] += absmode ? fabs(t[k]) : t[k];
        }
        if (op == 5) acc[0] += (absmode ? fabs(w[i]) : w[i]) * wend_a;   /* the particle itself */
        for (int k = 0; k < 4; ++k) out[4 * q + k] = acc[k];
    }
}

/*
 * Adjoints in FP64 over a given neighbour CSR (each row must list all
 * neighbours of the query; the relation is symmetric).
 *
 * GAUSS (op 1), loss L = sum_i g_i y_i:
 *   dL/dw_i = sum_j g_j exp(-s d_ij^2)
 *   dL/dx_i = sum_j (g_i w_j + g_j w_i) 2 s exp(-s d^2) dx_ij
 *   per-query share of dL/ds: -g_i sum_j w_j exp(-s d^2) d^2
 * LJ (op 2), loss L = sum_i g_i y_i with y_i the per-particle energy:
 *   dL/dx_i = sum_j 1/2 (g_i + g_j) C_ij dx_ij,
 *   C = eps (12 (sig/d)^12 - 6 (sig/d)^6) / d^2
 *   (with g = 1 this is minus the force on i).
 * out: float64[nq][4] position gradient; gw: float64[nq] (GAUSS) or NULL;
 * gs: float64[nq] (GAUSS) or NULL.  absmode != 0 sums term magnitudes
 * (the denominator of the error metric).
 */
void or_pair_grad(int op, int absmode, const double *prm, int dim,
                  const int *periodic,
                  const float *lo, const float *hi, int64_t n,
                  const double *pos64, const double *w, const double *g,
                  int64_t nq, const int64_t *queries, const int64_t *offsets,
                  const int32_t *idx, double *out, double *gw, double *gs) {
    box_t b;
    box_init(&b, dim, periodic, lo, hi, (float)prm[5]);
    const double s = prm[0], eps = prm[1], sig = prm[2];
    (void)n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t i = queries[q];
        const double *pi = pos64 + 4 * i;
        double acc[4] = {0, 0, 0, 0}, aw = 0, as = 0;
        for (int64_t e = offsets[q]; e < offsets[q + 1]; ++e) {
            int64_t j = idx[e];
            const double *pj = pos64 + 4 * j;
            double dx[3] = {0, 0, 0}, d2 = 0;
            for (int k = 0; k < dim; ++k) {
                dx[k] = sep64(&b, k, pi, pj);
                d2 += dx[k] * dx[k];
            }
            if (op == 1) {
                double kij = exp(-s * d2);
                if (absmode) {
                    double coef = (fabs(g[i] * w[j]) + fabs(g[j] * w[i])) * 2.0 * s * kij;
                    for (int k = 0; k < dim; ++k) acc[k] += coef * fabs(dx[k]);
                    aw += fabs(g[j]) * kij;
                    as += fabs(g[i] * w[j]) * kij * d2;
                } else {
                    double coef = (g[i] * w[j] + g[j] * w[i]) * 2.0 * s * kij;
                    for (int k = 0; k < dim; ++k) acc[k] += coef * dx[k];
                    aw += g[j] * kij;
                    as += -g[i] * w[j] * kij * d2;
                }
            } else if (op == 2) {
                double sr6 = pow(sig * sig / d2, 3);
                double C = absmode ? eps * (12.0 * sr6 * sr6 + 6.0 * sr6) / d2
                                   : eps * (12.0 * sr6 * sr6 - 6.0 * sr6) / d2;
                double coef = 0.5 * (g[i] + g[j]) * C;
                for (int k = 0; k < dim; ++k)
                    acc[k] += absmode ? fabs(coef * dx[k]) : coef * dx[k];
            }
        }
        for (int k = 0; k < 4; ++k) out[4 * q + k] = acc[k];
        if (gw) gw[q] = aw;
        if (gs) gs[q] = as;
    }
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
