/*
 * fkski CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow FP64 definitions of what the GPU path computes (the precompute uses OpenMP threads
 * over disjoint cell slabs with a fixed summation order, so results do not depend on them).  It shares no code
 * with the CUDA library and is used only by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline leg of bench.py.  Build with -ffp-contract=off so that the float sequence that
 * decides a cell index is evaluated exactly as written.
 *
 * Contents (each cites the passage it follows):
 *   or_cell_key_*     cell index + local coordinate of a point (Sec. 3, Def. 2: cubic
 *                     interpolation uses the 4 nearest nodes per axis; the boundary rule and the
 *                     exactly specified float sequence are this library's reading).
 *   or_keys_u         Keys' cubic-convolution kernel with a = -1/2 (cited in Def. 2's
 *                     discussion, Fig. 1: basis function centred at j, supported on [j-2, j+2)).
 *   or_precompute     sufficient statistics W^T W (as 7^d diagonals), W^T y, y^T y, and W^T z
 *                     for Rademacher probes (Sec. 3.1 "Precomputation"; Claim 2 for the band),
 *                     plus the stable cell sort (ties by input index) and segment offsets.
 *   or_w_rows         explicit rows of W (n x m, 4^d nonzeros per row), for the n-space CG oracle.
 *   or_rademacher     counter-based probe signs: SplitMix64 (Steele, Lea, Flood 2014; output
 *                     function as published by Vigna) evaluated at counter j*2^40 + i + 1.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

typedef struct {
    int d;
    int64_t M[3];
    double lo[3];
    double h[3];
} or_grid;

enum { OR_OK = 0, OR_E_INVALID = 1, OR_E_OUT_OF_GRID = 2, OR_E_NONFINITE = 3, OR_E_OOM = 4 };

/* ------------------------------------------------------------------ cell index of one coordinate
 * FP32 input.  s = (x - lo)/h is formed as an unevaluated pair of floats (error-free TwoSum and
 * FMA-based product, Dekker/Knuth), the cell is floor(s) of the pair's exact value, clamped to
 * [1, M-3] so that the stencil nodes c-1..c+2 exist; a point is inside iff 1 <= s <= M-2.
 * t32 is the float local coordinate (s_hi - c) + s_lo; t64 is the FP64 value (x - lo)/h - c. */
static void split_double(double v, float *hi, float *lo)
{
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
}

int or_cell_key_f32(float x, double lo, double h, int64_t M, int64_t *cell, float *t32, double *t64)
{
    if (!isfinite(x)) return OR_E_NONFINITE;
    float L1, L2, I1, I2;
    split_double(lo, &L1, &L2);
    split_double(1.0 / h, &I1, &I2);
    /* d = x - lo */
    float a = x, b = -L1;
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    e = e - L2;
    float d1 = s + e;
    float d2 = e - (d1 - s);
    /* s = d * (1/h) */
    float p = d1 * I1;
    float q = fmaf(d1, I1, -p);
    q = fmaf(d1, I2, q);
    q = fmaf(d2, I1, q);
    float s1 = p + q;
    float s2 = q - (s1 - p);
    float top = (float)(M - 2);
    int inside_lo = (s1 > 1.0f) || (s1 == 1.0f && s2 >= 0.0f);
    int inside_hi = (s1 < top) || (s1 == top && s2 <= 0.0f);
    if (!(inside_lo && inside_hi)) return OR_E_OUT_OF_GRID;
    float c = floorf(s1);
    if (s1 == c && s2 < 0.0f) c = c - 1.0f;
    int64_t ci = (int64_t)c;
    if (ci < 1) ci = 1;
    if (ci > M - 3) ci = M - 3;
    float u = s1 - (float)ci;
    *cell = ci;
    *t32 = u + s2;
    *t64 = ((double)x - lo) / h - (double)ci;
    return OR_OK;
}

/* FP64 input: s = (x - lo) * (1/h) in double, cell = floor(s) clamped to [1, M-3]. */
int or_cell_key_f64(double x, double lo, double h, int64_t M, int64_t *cell, double *t64)
{
    if (!isfinite(x)) return OR_E_NONFINITE;
    double ih = 1.0 / h;
    double s = (x - lo) * ih;
    if (!(s >= 1.0 && s <= (double)(M - 2))) return OR_E_OUT_OF_GRID;
    double c = floor(s);
    int64_t ci = (int64_t)c;
    if (ci < 1) ci = 1;
    if (ci > M - 3) ci = M - 3;
    *cell = ci;
    *t64 = s - (double)ci;
    return OR_OK;
}

/* ------------------------------------------------------------------ Keys cubic convolution
 * Keys (1981) kernel with a = -1/2:
 *   u(s) = 3/2|s|^3 - 5/2|s|^2 + 1              for |s| <= 1
 *   u(s) = -1/2|s|^3 + 5/2|s|^2 - 4|s| + 2      for 1 < |s| < 2
 *   u(s) = 0                                   otherwise.
 * A point at local coordinate t in [0,1] of cell c has weights u(t - (a - 1)) on the nodes
 * c - 1 + a, a = 0..3, i.e. u(1+t), u(t), u(1-t), u(2-t). */
double or_keys_u(double s)
{
    double as = fabs(s);
    if (as <= 1.0) return 1.5 * as * as * as - 2.5 * as * as + 1.0;
    if (as < 2.0) return -0.5 * as * as * as + 2.5 * as * as - 4.0 * as + 2.0;
    return 0.0;
}

void or_keys_weights(double t, double w[4])
{
    for (int a = 0; a < 4; ++a) w[a] = or_keys_u(t - (double)(a - 1));
}

/* ------------------------------------------------------------------ probes */
static uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Rademacher sign of probe j at point i: +1 or -1 from the top bit of the SplitMix64 output
 * at counter k = j*2^40 + i + 1 (the k-th value of the stream started at `seed`). */
double or_rademacher(uint64_t seed, int64_t j, int64_t i)
{
    uint64_t k = ((uint64_t)j << 40) + (uint64_t)i + 1ULL;
    return (splitmix64_at(seed, k) >> 63) ? -1.0 : 1.0;
}

void or_rademacher_fill(uint64_t seed, int64_t j, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_rademacher(seed, j, i);
}

/* ------------------------------------------------------------------ per-point stencil */
static int64_t ipow(int64_t b, int e)
{
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

/* Cell (per axis) and FP64 local coordinates of point i. */
static int point_cell(const or_grid *g, const void *X, int xdtype, int64_t n, int64_t i,
                      int64_t cell[3], double t[3])
{
    for (int k = 0; k < g->d; ++k) {
        int st;
        if (xdtype == 0) {
            float t32;
            st = or_cell_key_f32(((const float *)X)[k * n + i], g->lo[k], g->h[k], g->M[k],
                                 &cell[k], &t32, &t[k]);
        } else {
            st = or_cell_key_f64(((const double *)X)[k * n + i], g->lo[k], g->h[k], g->M[k],
                                 &cell[k], &t[k]);
        }
        if (st) return st;
    }
    return OR_OK;
}

/* Linear cell key: cells are indexed by c_k - 1 in [0, M_k - 4], C order (last axis fastest). */
static uint32_t cell_linear(const or_grid *g, const int64_t cell[3])
{
    int64_t key = 0;
    for (int k = 0; k < g->d; ++k) key = key * (g->M[k] - 3) + (cell[k] - 1);
    return (uint32_t)key;
}

int or_keys(const or_grid *g, const void *X, int xdtype, int64_t n, uint32_t *keys, float *t32)
{
    if (g->d < 1 || g->d > 3) return OR_E_INVALID;
    for (int64_t i = 0; i < n; ++i) {
        int64_t cell[3];
        double t[3];
        for (int k = 0; k < g->d; ++k) {
            int st;
            if (xdtype == 0) {
                float tf;
                st = or_cell_key_f32(((const float *)X)[k * n + i], g->lo[k], g->h[k], g->M[k],
                                     &cell[k], &tf, &t[k]);
                if (t32) t32[k * n + i] = tf;
            } else {
                st = or_cell_key_f64(((const double *)X)[k * n + i], g->lo[k], g->h[k], g->M[k],
                                     &cell[k], &t[k]);
                if (t32) t32[k * n + i] = (float)t[k];
            }
            if (st) return st;
        }
        keys[i] = cell_linear(g, cell);
    }
    return OR_OK;
}

/* Rows of W: for each point, 4^d node indices (C order over the grid) and FP64 weights.
 * Nonzero pattern: tensor product over axes of nodes c_k - 1 .. c_k + 2. */
int or_w_rows(const or_grid *g, const void *X, int xdtype, int64_t n, int64_t *cols, double *vals)
{
    const int d = g->d;
    const int64_t nnz = ipow(4, d);
    for (int64_t i = 0; i < n; ++i) {
        int64_t cell[3];
        double t[3], w[3][4];
        int st = point_cell(g, X, xdtype, n, i, cell, t);
        if (st) return st;
        for (int k = 0; k < d; ++k) or_keys_weights(t[k], w[k]);
        for (int64_t q = 0; q < nnz; ++q) {
            int64_t node = 0, rem = q;
            double wv = 1.0;
            int a[3];
            for (int k = d - 1; k >= 0; --k) { a[k] = (int)(rem % 4); rem /= 4; }
            for (int k = 0; k < d; ++k) {
                node = node * g->M[k] + (cell[k] - 1 + a[k]);
                wv *= w[k][a[k]];
            }
            cols[i * nnz + q] = node;
            vals[i * nnz + q] = wv;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ sufficient statistics
 * W^T W = sum_i w_i w_i^T, W^T y = sum_i y_i w_i, y^T y = sum_i y_i^2 (Sec. 3.1) in FP64.
 * W^T W is stored as its 7^d diagonals (Claim 2: entries are nonzero only for grid offsets delta
 * in {-3..3}^d):
 *   band[o * m + j] = (W^T W)[j, j + delta(o)],  o = sum_k (delta_k + 3) 7^(d-1-k).
 * Probe statistics: wtz[p * m + j] = (W^T z_p)[j] with z_p(i) = or_rademacher(seed, p, i).
 * Sort: perm is the stable sort of points by linear cell key (ties by input index);
 * offsets[c] .. offsets[c+1] is the segment of cell c.  Any output pointer may be NULL.
 *
 * Summation order (fixed, whatever the number of threads): points are summed in sorted order
 * (cell key, then input index).  Threads own disjoint slabs of cells: slab s holds the cells
 * whose first-axis index lies in [4s, 4s + 4), so its points touch grid nodes [4s, 4s + 6] on
 * that axis; the even slabs run first (their node ranges are disjoint, so they run in
 * parallel), then the odd slabs.  Every entry therefore receives its terms in one order: the
 * even slab's points in sorted order, then the odd slab's.  y^T y is summed per slab and the
 * slab sums are added in slab order. */
static void point_terms(const or_grid *g, const int64_t cell[3], const double t[3], int64_t node[64],
                        double wv[64], int aidx[64][3])
{
    const int d = g->d;
    const int64_t nnz = ipow(4, d);
    double w[3][4];
    for (int k = 0; k < d; ++k) or_keys_weights(t[k], w[k]);
    for (int64_t q = 0; q < nnz; ++q) {
        int64_t rem = q, nd = 0;
        double v = 1.0;
        int a[3] = {0, 0, 0};
        for (int k = d - 1; k >= 0; --k) { a[k] = (int)(rem % 4); rem /= 4; }
        for (int k = 0; k < d; ++k) {
            nd = nd * g->M[k] + (cell[k] - 1 + a[k]);
            v *= w[k][a[k]];
            aidx[q][k] = a[k];
        }
        node[q] = nd;
        wv[q] = v;
    }
}

/* Accumulate the points perm[b..e) (one slab, sorted order) into the statistics; returns the slab's
 * sum of y_i^2. */
static double slab_sums(const or_grid *g, const void *X, int xdtype, const void *y, int64_t n, int nprobe,
                        uint64_t seed, const int64_t *perm, int64_t b, int64_t e, int64_t m,
                        double *band, double *wty, double *wtz)
{
    const int d = g->d;
    const int64_t nnz = ipow(4, d);
    double yy = 0.0;
    for (int64_t s = b; s < e; ++s) {
        const int64_t i = perm[s];
        int64_t cell[3];
        double t[3];
        point_cell(g, X, xdtype, n, i, cell, t);  /* checked when the keys were formed */
        const double yi = xdtype == 0 ? (double)((const float *)y)[i] : ((const double *)y)[i];
        yy += yi * yi;
        int64_t node[64];
        double wv[64];
        int aidx[64][3];
        point_terms(g, cell, t, node, wv, aidx);
        if (band) {
            for (int64_t qa = 0; qa < nnz; ++qa) {
                for (int64_t qb = 0; qb < nnz; ++qb) {
                    int64_t o = 0;
                    for (int k = 0; k < d; ++k) o = o * 7 + (aidx[qb][k] - aidx[qa][k] + 3);
                    band[o * m + node[qa]] += wv[qa] * wv[qb];
                }
            }
        }
        if (wty)
            for (int64_t q = 0; q < nnz; ++q) wty[node[q]] += yi * wv[q];
        if (wtz)
            for (int p = 0; p < nprobe; ++p) {
                const double z = or_rademacher(seed, p, i);
                for (int64_t q = 0; q < nnz; ++q) wtz[(int64_t)p * m + node[q]] += z * wv[q];
            }
    }
    return yy;
}

int or_precompute(const or_grid *g, const void *X, int xdtype, const void *y, int64_t n,
                  int nprobe, uint64_t seed, uint32_t *keys, int64_t *perm, int64_t *offsets,
                  double *band, double *wty, double *yty, double *wtz)
{
    const int d = g->d;
    if (d < 1 || d > 3 || n < 1) return OR_E_INVALID;
    int64_t m = 1, ncell = 1;
    for (int k = 0; k < d; ++k) {
        if (g->M[k] < 4 || !(g->h[k] > 0.0)) return OR_E_INVALID;
        m *= g->M[k];
        ncell *= g->M[k] - 3;
    }
    const int64_t nband = ipow(7, d);
    uint32_t *kk = keys ? keys : (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    int64_t *pp = perm ? perm : (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *cnt = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    if (!kk || !pp || !cnt) {
        if (!keys) free(kk);
        if (!perm) free(pp);
        free(cnt);
        return OR_E_OOM;
    }
    /* cell keys (independent per point); the error reported is the first point's in input order */
    int64_t bad_i = n;
    int bad_st = OR_OK;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t cell[3];
        double t[3];
        int st = point_cell(g, X, xdtype, n, i, cell, t);
        if (st == OR_OK) {
            const double yi = xdtype == 0 ? (double)((const float *)y)[i] : ((const double *)y)[i];
            if (!isfinite(yi)) st = OR_E_NONFINITE;
        }
        if (st != OR_OK) {
#pragma omp critical
            if (i < bad_i) { bad_i = i; bad_st = st; }
            kk[i] = 0;
        } else {
            kk[i] = cell_linear(g, cell);
        }
    }
    int rc = bad_st;
    if (rc == OR_OK) {
        /* stable counting sort by key */
        for (int64_t i = 0; i < n; ++i) cnt[kk[i] + 1] += 1;
        for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
        if (offsets) memcpy(offsets, cnt, sizeof(int64_t) * (size_t)(ncell + 1));
        {
            int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
            if (!pos) rc = OR_E_OOM;
            else {
                memcpy(pos, cnt, sizeof(int64_t) * (size_t)(ncell + 1));
                for (int64_t i = 0; i < n; ++i) pp[pos[kk[i]]++] = i;
                free(pos);
            }
        }
    }
    if (rc == OR_OK && (band || wty || wtz || yty)) {
        if (band) memset(band, 0, sizeof(double) * (size_t)(nband * m));
        if (wty) memset(wty, 0, sizeof(double) * (size_t)m);
        if (wtz && nprobe > 0) memset(wtz, 0, sizeof(double) * (size_t)(nprobe * m));
        const int64_t per0 = ncell / (g->M[0] - 3);   /* cells per first-axis index */
        const int64_t nslab = (g->M[0] - 3 + 3) / 4;
        double *yslab = (double *)calloc((size_t)nslab, sizeof(double));
        if (!yslab) rc = OR_E_OOM;
        for (int phase = 0; phase < 2 && rc == OR_OK; ++phase) {
#pragma omp parallel for schedule(dynamic, 1)
            for (int64_t sl = phase; sl < nslab; sl += 2) {
                const int64_t c0 = 4 * sl, c1 = c0 + 4 < g->M[0] - 3 ? c0 + 4 : g->M[0] - 3;
                yslab[sl] = slab_sums(g, X, xdtype, y, n, nprobe, seed, pp, cnt[c0 * per0], cnt[c1 * per0], m,
                                      band, wty, wtz);
            }
        }
        if (rc == OR_OK && yty) {
            double yy = 0.0;
            for (int64_t sl = 0; sl < nslab; ++sl) yy += yslab[sl];
            *yty = yy;
        }
        free(yslab);
    }
    free(cnt);
    if (!keys) free(kk);
    if (!perm) free(pp);
    return rc;
}

/* Threads the oracle may use (OpenMP); 0 leaves the OpenMP default. */
void or_set_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Posterior mean at test points: mu(x*) = w_{x*}^T v (Def. 1 mean; Fact 2 mean with v = z_bar). */
int or_predict(const or_grid *g, const double *v, const void *Xs, int xdtype, int64_t ns,
               double *mu)
{
    const int d = g->d;
    const int64_t nnz = ipow(4, d);
    for (int64_t i = 0; i < ns; ++i) {
        int64_t cell[3];
        double t[3], w[3][4];
        int st = point_cell(g, Xs, xdtype, ns, i, cell, t);
        if (st) return st;
        for (int k = 0; k < d; ++k) or_keys_weights(t[k], w[k]);
        double acc = 0.0;
        for (int64_t q = 0; q < nnz; ++q) {
            int64_t rem = q, nd = 0;
            double wv = 1.0;
            int a[3] = {0, 0, 0};
            for (int k = d - 1; k >= 0; --k) { a[k] = (int)(rem % 4); rem /= 4; }
            for (int k = 0; k < d; ++k) {
                nd = nd * g->M[k] + (cell[k] - 1 + a[k]);
                wv *= w[k][a[k]];
            }
            acc += wv * v[nd];
        }
        mu[i] = acc;
    }
    return OR_OK;
}
