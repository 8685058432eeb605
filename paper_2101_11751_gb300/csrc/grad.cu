// Log marginal likelihood (Def. 1) and its gradient w.r.t. (l_1..l_d, s, sigma^2) from the
// sufficient statistics only.
//
//   L = -1/2 [ logdet A + y^T A^{-1} y + n log 2 pi ],   A = W K_G W^T + sigma^2 I.
// Solves: batched factorized CG (Alg. 3, x0 = 0) on [y, z_1..z_T], z_p the Rademacher probes
// whose W^T z_p the precompute accumulated.  From the compressed solution x = W x_hat + c^x b:
//   W^T x = W^T W x_hat + c^x W^T b     (x_hat in FP64, one FP64 SpMV at the end)
//   b^T x = (W^T b)^T x_hat + c^x b^T b
// logdet A by stochastic Lanczos quadrature: each probe's CG coefficients give the Lanczos
// tridiagonal T_p (T[0,0] = 1/a_0, T[i,i] = 1/a_i + b_{i-1}/a_{i-1}, T[i,i+1] = sqrt(b_i)/a_i) and
//   z_p^T log(A) z_p ~ ||z_p||^2 e_1^T log(T_p) e_1,
// evaluated from the eigen-decomposition of T_p (implicit-shift QL, first eigenvector row only).
// Gradient (Hutchinson traces with the same probes):
//   dL/dtheta   = 1/2 a^T dK a - 1/2 mean_p (W^T x_p)^T dK (W^T z_p),  a = W^T A^{-1} y
//   dL/dsigma^2 = 1/2 ||A^{-1} y||^2 - 1/2 mean_p z_p^T x_p,
//   ||A^{-1} y||^2 = (y^T y - 2 (W^T y)^T K a + (K a)^T W^T W (K a)) / sigma^4
// since A^{-1} y = (y - W K a) / sigma^2.
#include "fkski_internal.cuh"

#include <algorithm>
#include <thread>
#include <vector>

namespace fk {

int grad_solve(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, int dtype, void *sol, double *a64,
               double *zx, int *iters, double *res, int *status, cudaStream_t s);

// The solve workspace layout is private to solve.cu; grad.cu reaches it through these.
struct GradView {
    double *S;        // per-rhs fields (solve.cu enum)
    double *hist_a;   // alpha history [k * R + r]
    double *hist_b;   // beta history
    int *iters;       // device per-rhs counts
    KgOp *kg;
};
int grad_view(fkski_stats *st, int dtype, GradView *gv);
int grad_sol_buffer(fkski_stats *st, size_t bytes, void **p);
void grad_sol_mark(fkski_stats *st, int valid, const fkski_kernel *kern, int dtype);
int grad_sol_valid(fkski_stats *st, const fkski_kernel *kern, int dtype);
constexpr int GF_RHO0 = 7;  // must match solve.cu's field enum
int spmv_for_grad(fkski_stats *st, const void *x, void *u, int R, int dtype, cudaStream_t s);

// ------------------------------------------------------------------ SLQ
// Per probe, the implicit QL iteration on the k x k Lanczos tridiagonal (FP64) carrying the first
// row of the eigenvector matrix; est[p] = rho0 sum_l z_l^2 log lam_l.  It runs on the host cores,
// one thread per probe: the sweep is a sequential chain of FP64 divides and square roots, O(k^2)
// for k CG steps (about 1.5e8 rotations at k = 12,000), which a single GPU thread on GB300's FP64
// pipe runs tens of times slower than one host core.  Only the CG coefficients (k per probe) move.
constexpr int SLQ_MAXK = 65536;

// e_1^T log(T) e_1 for the symmetric tridiagonal T (diagonal dg[0..k), couplings of[i] between
// i and i+1, z = e_1 on entry): implicit-shift QL on (dg, of), rotating the first row z of the
// eigenvector matrix along; Ritz values are clamped at sig2 (the spectrum of A starts there).
// dg, of and z are overwritten.  Returns the quadrature; *fail when QL did not converge or a
// Ritz value is not finite.
static double tridiag_e1_log(double *dg, double *of, double *z, int k, double sig2, int *fail_out) {
    const double eps = 2.220446049250313e-16;
    int fail = 0;
    for (int l = 0; l < k; ++l) {
        for (int guard = 0; guard < 60; ++guard) {
            // smallest m >= l with a negligible coupling below it
            int mm = l;
            while (mm < k - 1 && std::fabs(of[mm]) > eps * (std::fabs(dg[mm]) + std::fabs(dg[mm + 1]))) ++mm;
            if (mm == l) break;
            if (guard == 59) { fail = 1; break; }
            // Wilkinson-type shift from the leading 2x2 block at l
            double gq = (dg[l + 1] - dg[l]) / (2.0 * of[l]);
            double rr = std::hypot(gq, 1.0);
            gq = dg[mm] - dg[l] + of[l] / (gq + (gq >= 0.0 ? rr : -rr));
            double sn = 1.0, cs = 1.0, pp = 0.0;
            int i = mm - 1;
            bool early = false;
            for (; i >= l; --i) {
                const double f = sn * of[i], b = cs * of[i];
                rr = std::hypot(f, gq);
                of[i + 1] = rr;
                if (rr == 0.0) {
                    dg[i + 1] -= pp;
                    of[mm] = 0.0;
                    early = true;
                    break;
                }
                sn = f / rr;
                cs = gq / rr;
                gq = dg[i + 1] - pp;
                rr = (dg[i] - gq) * sn + 2.0 * cs * b;
                pp = sn * rr;
                dg[i + 1] = gq + pp;
                gq = cs * rr - b;
                const double zf = z[i + 1];
                z[i + 1] = sn * z[i] + cs * zf;
                z[i] = cs * z[i] - sn * zf;
            }
            if (early) continue;
            dg[l] -= pp;
            of[l] = gq;
            of[mm] = 0.0;
        }
    }
    double acc = 0.0;
    for (int i = 0; i < k; ++i) {
        if (!std::isfinite(dg[i])) fail = 1;
        else acc += z[i] * z[i] * std::log(std::fmax(dg[i], sig2));
    }
    *fail_out = fail;
    return acc;
}

// The Lanczos tridiagonal of probe r from its CG coefficients (T[0,0] = 1/a_0,
// T[i,i] = 1/a_i + b_{i-1}/a_{i-1}, T[i,i+1] = sqrt(b_i)/a_i), then its quadrature.
// A = W K W^T + sigma^2 I has spectrum in [sigma^2, inf), so a Ritz value below sigma^2 (left by
// rounding in the Krylov recurrences) is clamped to sigma^2.
static double slq_probe(const double *ha, const double *hb, int R, int r, int k, double sig2, int *fail) {
    *fail = 0;
    if (k == 0) return 0.0;
    std::vector<double> dg(k), of(k), z(k);
    for (int i = 0; i < k; ++i) {
        const double a = ha[(int64_t)i * R + r];
        double di = 1.0 / a;
        if (i > 0) di += hb[(int64_t)(i - 1) * R + r] / ha[(int64_t)(i - 1) * R + r];
        dg[i] = di;
        of[i] = (i + 1 < k) ? std::sqrt(hb[(int64_t)i * R + r]) / a : 0.0;
        z[i] = (i == 0) ? 1.0 : 0.0;
    }
    return tridiag_e1_log(dg.data(), of.data(), z.data(), k, sig2, fail);
}

// dots of row pairs: out[r] = sum_i a[r][i] b[r][i]; per-block FP64 partials then a fixed-order sum
template <typename T>
__global__ void __launch_bounds__(256) k_rowdots(const T *__restrict__ a, const T *__restrict__ b, int64_t m, int R,
                                                 double *__restrict__ part) {
    __shared__ double sh[8];
    for (int r = 0; r < R; ++r) {
        T acc = T(0);
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
            acc = fma(a[(int64_t)r * m + j], b[(int64_t)r * m + j], acc);
        double dv = (double)acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dv += __shfl_xor_sync(0xFFFFFFFFu, dv, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dv;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += sh[w];
            part[(int64_t)blockIdx.x * R + r] = s;
        }
        __syncthreads();
    }
}

__global__ void k_sum_rows(const double *__restrict__ part, int nb, int R, double *__restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * R + r];
    out[r] = s;
}

constexpr int RD_BLOCKS = 304;

template <typename T>
static int rowdots(const T *a, const T *b, int64_t m, int R, double *part, double *out, cudaStream_t s) {
    k_rowdots<T><<<RD_BLOCKS, 256, 0, s>>>(a, b, m, R, part);
    FK_LAUNCH();
    k_sum_rows<<<(unsigned)cdiv(R, 64), 64, 0, s>>>(part, RD_BLOCKS, R, out);
    FK_LAUNCH();
    return FKSKI_OK;
}

// Forward scalars.  fs layout: [0] L, [1] logdet, [2] quad, [3 + p] z_p^T x_p (p >= 1).
// zx[r] = b_r^T x_r from the solve (r = 0: y^T A^{-1} y).
__global__ void k_loglik_assemble(const double *__restrict__ S, const double *__restrict__ zx,
                                  const double *__restrict__ est, int R, double n, double *__restrict__ fs) {
    if (threadIdx.x != 0) return;
    const double quad = zx[0];
    double ld = 0.0;
    for (int p = 1; p < R; ++p) ld += est[p - 1];
    ld /= (double)(R - 1);
    fs[0] = -0.5 * (ld + quad + n * log(2.0 * 3.14159265358979323846));
    fs[1] = ld;
    fs[2] = quad;
    for (int p = 1; p < R; ++p) fs[3 + p] = zx[p];
}

// grad[t] for kernel params from dots dd[t*R + r] = sol[r] . dK_t src[r]
__global__ void k_grad_assemble(const double *__restrict__ dd, int nth, int R, const double *__restrict__ fs,
                                const double *__restrict__ s2dots, double yty, double sig2, double *__restrict__ grad) {
    if (threadIdx.x != 0) return;
    const int T = R - 1;
    for (int t = 0; t < nth; ++t) {
        double tr = 0.0;
        for (int p = 1; p < R; ++p) tr += dd[t * R + p];
        grad[t] = 0.5 * dd[t * R + 0] - 0.5 * tr / (double)T;
    }
    // sigma^2: s2dots[0] = (W^T y).(K a), s2dots[1] = (K a).(W^T W K a)
    const double zz = (yty - 2.0 * s2dots[0] + s2dots[1]) / (sig2 * sig2);
    double tr = 0.0;
    for (int p = 1; p < R; ++p) tr += fs[3 + p];
    grad[nth] = 0.5 * zz - 0.5 * tr / (double)T;
}

template <typename T>
__global__ void k_widen(const T *__restrict__ a, double *__restrict__ out, int64_t m) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (double)a[e];
}

template <typename T>
__global__ void k_copy_rows(const T *__restrict__ a, const T *__restrict__ wtz, int64_t m, int R, T *__restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = e < m ? a[e] : wtz[e - m];
}

// ------------------------------------------------------------------ forward
// Slot kept between forward and backward (the stats' solution buffer):
//   sol : R x m  W^T x_r in the solve precision (row 0 is a = W^T A^{-1} y)
//   a64 : m      a in FP64 (for the sigma^2 terms)
//   fs  : 3 + R + 64 forward scalars (see k_loglik_assemble), then zx (R) and partials
template <typename T>
struct Slot {
    T *sol;
    double *a64, *fs, *zx, *part;
};

template <typename T>
static int slot_get(fkski_stats *st, int R, int64_t m, bool alloc, Slot<T> &sl) {
    const size_t sol_bytes = sizeof(T) * (size_t)R * m;
    const size_t a_off = (sol_bytes + 255) / 256 * 256;
    const size_t need = a_off + sizeof(double) * ((size_t)m + 3 + R + 64 + R + (size_t)RD_BLOCKS * R + 16);
    void *slot;
    FK_TRY(grad_sol_buffer(st, alloc ? need : 0, &slot));
    sl.sol = (T *)slot;
    sl.a64 = (double *)((char *)slot + a_off);
    sl.fs = sl.a64 + m;
    sl.zx = sl.fs + 3 + R + 64;
    sl.part = sl.zx + R;
    return FKSKI_OK;
}

template <typename T>
static int forward_typed(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, double *L, fkski_info *info,
                         cudaStream_t s) {
    const int R = 1 + st->nprobes;
    const int64_t m = st->m;
    const int dt = dtype_of<T>();
    Slot<T> sl;
    FK_TRY(slot_get<T>(st, R, m, true, sl));
    std::vector<int> it(R, 0);
    std::vector<double> res(R, 0.0);
    int status = FKSKI_OK;
    FK_TRY(grad_solve(st, kern, o, dt, sl.sol, sl.a64, sl.zx, it.data(), res.data(), &status, s));
    GradView gv;
    FK_TRY(grad_view(st, dt, &gv));
    double *est = sl.part;  // R doubles of scratch
    int kmax = 0;
    for (int r = 1; r < R; ++r) kmax = std::max(kmax, it[r]);
    if (kmax > SLQ_MAXK) return FKSKI_E_UNSUPPORTED;
    // CG coefficients and rho0 to the host; one thread per probe
    std::vector<double> ha((size_t)std::max(kmax, 1) * R), hb((size_t)std::max(kmax, 1) * R), hS((size_t)R);
    FK_CUDA(cudaMemcpyAsync(ha.data(), gv.hist_a, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaMemcpyAsync(hb.data(), gv.hist_b, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaMemcpyAsync(hS.data(), gv.S + (size_t)GF_RHO0 * R, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaStreamSynchronize(s));
    std::vector<double> hest((size_t)R, 0.0);
    std::vector<int> hfail((size_t)R, 0);
    {
        std::vector<std::thread> pool;
        for (int r = 1; r < R; ++r)
            pool.emplace_back([&, r]() {
                hest[r - 1] = hS[r] * slq_probe(ha.data(), hb.data(), R, r, it[r], kern->noise_var, &hfail[r]);
            });
        for (auto &t : pool) t.join();
    }
    int hst = 0;
    for (int r = 1; r < R; ++r)
        if (hfail[r]) hst |= ST_BREAKDOWN;
    FK_CUDA(cudaMemcpyAsync(est, hest.data(), sizeof(double) * (R - 1), cudaMemcpyHostToDevice, s));
    k_loglik_assemble<<<1, 32, 0, s>>>(gv.S, sl.zx, est, R, (double)st->n, sl.fs);
    FK_LAUNCH();
    FK_CUDA(cudaMemcpyAsync(L, sl.fs, sizeof(double), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaStreamSynchronize(s));
    if (info) {
        info->iters = 0;
        info->rel_residual = 0.0;
        for (int r = 0; r < R && r < 65; ++r) {
            info->iters_rhs[r] = it[r];
            info->iters = std::max(info->iters, it[r]);
            info->rel_residual = std::max(info->rel_residual, res[r]);
        }
        info->status = status;
    }
    const bool keep = 2 * sizeof(T) * (size_t)R * m <= o->iterate_budget_bytes;
    grad_sol_mark(st, keep ? 1 : 0, kern, dt);
    if (hst & ST_BREAKDOWN) return FKSKI_E_BREAKDOWN;
    return status;
}

// ------------------------------------------------------------------ backward
template <typename T>
static int backward_typed(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, double *grad,
                          fkski_info *info, cudaStream_t s) {
    const int dt = dtype_of<T>();
    if (!grad_sol_valid(st, kern, dt)) {
        double Ltmp;
        fkski_opts o2 = *o;
        o2.iterate_budget_bytes = (size_t)-1;  // keep for this backward pass
        const int rc = forward_typed<T>(st, kern, &o2, &Ltmp, info, s);
        if (rc != FKSKI_OK && rc != FKSKI_E_NOT_CONVERGED) return rc;
    }
    const int R = 1 + st->nprobes;
    const int64_t m = st->m;
    const int d = st->d;
    GradView gv;
    FK_TRY(grad_view(st, dt, &gv));
    Slot<T> sl;
    FK_TRY(slot_get<T>(st, R, m, false, sl));
    const void *bandv, *wtyv, *wtzv;
    FK_TRY(stats_band_as(st, dt, &bandv, &wtyv, &wtzv, s));
    const T *wty = (const T *)wtyv, *wtz = (const T *)wtzv;
    T *src, *dK;
    double *dd, *v64;
    const size_t sol_bytes = sizeof(T) * (size_t)R * m;
    FK_TRY(pool_alloc((void **)&src, 2 * sol_bytes, s));
    dK = src + (size_t)R * m;
    FK_TRY(pool_alloc((void **)&v64, sizeof(double) * 3 * m, s));
    FK_TRY(pool_alloc((void **)&dd, sizeof(double) * ((d + 1) * R + 8 + 8), s));
    double *s2dots = dd + (d + 1) * R;
    double *dgrad = s2dots + 4;
    const unsigned gb = (unsigned)std::min<int64_t>(cdiv((int64_t)R * m, 256), 152 * 8);
    // src = [a, W^T z_1, ..., W^T z_T]
    k_copy_rows<T><<<gb, 256, 0, s>>>(sl.sol, wtz, m, R, src);
    FK_LAUNCH();
    KgOp *kg = gv.kg;
    for (int t = 0; t <= d; ++t) {
        FK_TRY(kgop_set(kg, kern, t, s));
        FK_TRY(kgop_apply(kg, src, dK, R, nullptr, 0.0, s));
        FK_TRY(rowdots<T>(sl.sol, dK, m, R, sl.part, dd + t * R, s));
    }
    FK_TRY(kgop_set(kg, kern, -1, s));
    // sigma^2 terms in FP64: v = K_G a, u = W^T W v; (W^T y).v and v.u
    double *u64 = v64 + m, *g64 = v64 + 2 * m;
    KgOp *kg64;
    FK_TRY(kgop_create(&st->grid, FKSKI_F64, &kg64));
    int rc = kgop_set(kg64, kern, -1, s);
    if (rc == FKSKI_OK) rc = kgop_apply(kg64, sl.a64, v64, 1, nullptr, 0.0, s);
    if (rc == FKSKI_OK) rc = spmv_for_grad(st, v64, u64, 1, FKSKI_F64, s);
    if (rc == FKSKI_OK) {
        k_widen<T><<<gb, 256, 0, s>>>(wty, g64, m);
        rc = cudaGetLastError() == cudaSuccess ? FKSKI_OK : FKSKI_E_CUDA;
    }
    if (rc == FKSKI_OK) rc = rowdots<double>(g64, v64, m, 1, sl.part, s2dots, s);
    if (rc == FKSKI_OK) rc = rowdots<double>(v64, u64, m, 1, sl.part, s2dots + 1, s);
    cudaStreamSynchronize(s);
    kgop_destroy(kg64);
    if (rc != FKSKI_OK) return rc;
    k_grad_assemble<<<1, 32, 0, s>>>(dd, d + 1, R, sl.fs, s2dots, st->yty, kern->noise_var, dgrad);
    FK_LAUNCH();
    FK_CUDA(cudaMemcpyAsync(grad, dgrad, sizeof(double) * (d + 2), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaFreeAsync(src, s));
    FK_CUDA(cudaFreeAsync(v64, s));
    FK_CUDA(cudaFreeAsync(dd, s));
    FK_CUDA(cudaStreamSynchronize(s));
    (void)o;
    return FKSKI_OK;
}

static int check_grad_args(fkski_stats *st, const fkski_kernel *kern, fkski_opts *o, const fkski_opts *opts) {
    if (!st || !kern) return FKSKI_E_INVALID_ARG;
    if (opts) *o = *opts; else fkski_default_opts(o);
    if (st->nprobes < 1) return FKSKI_E_INVALID_ARG;
    if (!(kern->noise_var > 0.0)) return FKSKI_E_INVALID_ARG;
    if (o->maxiter < 1 || o->maxiter > SLQ_MAXK) return FKSKI_E_INVALID_ARG;
    if (o->precision != FKSKI_MIXED && o->precision != FKSKI_DOUBLE && o->precision != FKSKI_FP32)
        return FKSKI_E_INVALID_ARG;
    return FKSKI_OK;
}

int loglik_forward_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, double *L, fkski_info *info,
                        cudaStream_t s) {
    fkski_opts o;
    FK_TRY(check_grad_args(st, kern, &o, opts));
    if (!L) return FKSKI_E_INVALID_ARG;
    if (info) memset(info, 0, sizeof(*info));
    if (o.precision == FKSKI_DOUBLE) return forward_typed<double>(st, kern, &o, L, info, s);
    if (o.precision == FKSKI_FP32) return forward_typed<float>(st, kern, &o, L, info, s);
    return forward_typed<dfl>(st, kern, &o, L, info, s);
}

int loglik_backward_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, double *grad,
                         fkski_info *info, cudaStream_t s) {
    fkski_opts o;
    FK_TRY(check_grad_args(st, kern, &o, opts));
    if (!grad) return FKSKI_E_INVALID_ARG;
    if (o.precision == FKSKI_DOUBLE) return backward_typed<double>(st, kern, &o, grad, info, s);
    if (o.precision == FKSKI_FP32) return backward_typed<float>(st, kern, &o, grad, info, s);
    return backward_typed<dfl>(st, kern, &o, grad, info, s);
}


// log det A by stochastic Lanczos quadrature over the precompute's probes, each with k steps of
// EFLA (App. B) -- the factorized-Lanczos alternative to the CG-coefficient SLQ of the
// log-likelihood: logdet ~ mean_p ||z_p||^2 e_1^T log(T_p) e_1.
int logdet_lanczos_impl(fkski_stats *st, const fkski_kernel *kern, int k, double *logdet, double *terms,
                        fkski_info *info, cudaStream_t s) {
    if (!st || !kern || !logdet || k < 1) return FKSKI_E_INVALID_ARG;
    if (st->nprobes < 1) return FKSKI_E_INVALID_ARG;
    if (!(kern->noise_var > 0.0)) return FKSKI_E_INVALID_ARG;
    if (info) memset(info, 0, sizeof(*info));
    double sum = 0.0;
    int hst = 0;
    for (int p = 0; p < st->nprobes; ++p) {
        std::vector<double> dg, of;
        FK_TRY(efla_probe_tridiag(st, kern, k, p, dg, of, info, s));
        const int kk = (int)dg.size();
        std::vector<double> z((size_t)std::max(kk, 1), 0.0);
        z[0] = 1.0;
        int fail = 0;
        const double t = kk > 0 ? st->ztz[p] * tridiag_e1_log(dg.data(), of.data(), z.data(), kk, kern->noise_var, &fail)
                                : 0.0;
        if (fail) hst |= ST_BREAKDOWN;
        if (terms) terms[p] = t;
        sum += t;
    }
    *logdet = sum / st->nprobes;
    if (hst & ST_BREAKDOWN) return FKSKI_E_BREAKDOWN;
    return FKSKI_OK;
}
}  // namespace fk
