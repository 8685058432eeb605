// m-space solves from the sufficient statistics (Sec. 4, App. B) and posterior-mean prediction.
//
// B(x) = [(K_G W^T W + sigma^2 I) x, W^T W x] is one banded SpMV (Claim 2, 7^d diagonals) feeding
// one K_G application (kg.cu).  Two factorized CG variants share it:
//   Alg. 5 (simplified EFCG): r0 in span(W) via x0 = y / sigma^2; returns W^T x directly.
//   Alg. 3 (EFCG, x0 = 0): compressed iterates v = W v_hat + c v0 with scalar coefficients;
//     batched over right-hand sides [y, z_1..z_T] so every B(x) reads the band once.
// Vectors are FP32 (MIXED) or FP64 (DOUBLE); inner products are summed in FP32 inside a warp and
// in FP64 across warps and blocks, always in the same order (deterministic).  All scalars live in
// device memory; iterations run as a captured CUDA graph of `check_every` steps with a device
// convergence flag tested by the host between graph launches.
#include "fkski_internal.cuh"

#include <algorithm>
#include <vector>

namespace fk {

constexpr int CG_T = 256;

// per-rhs scalar fields (double S[F * R + r])
enum {
    F_GAMMA = 0, F_GNEW, F_ALPHA, F_BETA, F_CR, F_CP, F_CX, F_RHO0, F_EPS, F_GKG, F_DELTA, F_RES, NF
};

struct CgCtl {
    int iter;      // completed alpha steps
    int all_done;
    int status;    // ST_* bits
    int maxiter;
    int R;
    int pad[3];
    double sig2;
};

struct BandOffs {
    int off[343];
};

// ------------------------------------------------------------------ reductions
// Block partial of a per-thread FP32 value: FP32 warp tree, FP64 across warps.
template <typename T>
__device__ __forceinline__ double block_sum(T v, double *sh) {
    float f = (float)v;
    double dv = 0.0;
    if (sizeof(T) == 4) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xFFFFFFFFu, f, o);
        dv = (double)f;
    } else {
        dv = (double)v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dv += __shfl_xor_sync(0xFFFFFFFFu, dv, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = dv;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    __syncthreads();
    return s;  // valid in thread 0
}

// Sum partials part[b * NQ * R + r * NQ + q] over b in fixed order; one warp per (r, q).
__device__ __forceinline__ double warp_sum_partials(const double *part, int nparts, int R, int NQ, int r, int q) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nparts; b += 32) s += part[(int64_t)b * NQ * R + r * NQ + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    return s;
}

// ------------------------------------------------------------------ band SpMV
// u[r][j] = sum_o band[o][j] * x[r][j + off(o)]  (entries whose neighbour is off-grid are zero,
// so the neighbour index is only clamped to stay in memory).  Optional partial dots per rhs:
// q0 = u.x, q1 = x.g (g per rhs, rhs-major).
template <typename T, int RB>
__global__ void __launch_bounds__(CG_T) k_band_spmv(const T *__restrict__ band, int nband, const T *__restrict__ x,
                                                     T *__restrict__ u, int64_t m, int R, BandOffs offs,
                                                     double *__restrict__ part, int NQ, const T *__restrict__ g,
                                                     const CgCtl *__restrict__ ctl, int Rtot, int r0) {
    if (ctl && ctl->all_done) return;
    __shared__ double sh[CG_T / 32];
    T dq0[RB], dq1[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) dq0[k] = dq1[k] = T(0);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        T acc[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) acc[k] = T(0);
        for (int o = 0; o < nband; ++o) {
            const T b = band[(int64_t)o * m + j];
            int64_t nb = j + offs.off[o];
            nb = nb < 0 ? 0 : (nb >= m ? m - 1 : nb);
#pragma unroll
            for (int k = 0; k < RB; ++k)
                if (k < R) acc[k] = fma(b, x[(int64_t)k * m + nb], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < RB; ++k)
            if (k < R) {
                u[(int64_t)k * m + j] = acc[k];
                if (part) {
                    const T xv = x[(int64_t)k * m + j];
                    dq0[k] = fma(acc[k], xv, dq0[k]);
                    if (g) dq1[k] = fma(xv, g[(int64_t)k * m + j], dq1[k]);
                }
            }
    }
    if (!part) return;
    for (int k = 0; k < R && k < RB; ++k) {
        const double s0 = block_sum<T>(dq0[k], sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + 0] = s0;
        if (NQ > 1) {
            const double s1 = block_sum<T>(dq1[k], sh);
            if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + 1] = s1;
        }
    }
}

static BandOffs make_offs(const fkski_grid &g) {
    BandOffs bo;
    memset(&bo, 0, sizeof(bo));
    const int d = g.d;
    int64_t stride[3] = {1, 1, 1};
    for (int k = d - 2; k >= 0; --k) stride[k] = stride[k + 1] * g.M[k + 1];
    const int nb = (int)ipow(7, d);
    for (int o = 0; o < nb; ++o) {
        int rem = o;
        int64_t off = 0;
        for (int k = d - 1; k >= 0; --k) {
            off += (int64_t)((rem % 7) - 3) * stride[k];
            rem /= 7;
        }
        bo.off[o] = (int)off;
    }
    return bo;
}

static int grid_blocks(int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(work, CG_T), 152 * 4)); }

template <typename T>
static int launch_spmv(const T *band, const fkski_grid &g, const T *x, T *u, int64_t m, int R, double *part, int NQ,
                       const T *gv, const CgCtl *ctl, int nblocks, cudaStream_t s) {
    const BandOffs bo = make_offs(g);
    const int nb = (int)ipow(7, g.d);
    for (int r0 = 0; r0 < R; r0 += 32) {
        const int Rb = std::min(32, R - r0);
        const T *xb = x + (int64_t)r0 * m;
        T *ub = u + (int64_t)r0 * m;
        const T *gb = gv ? gv + (int64_t)r0 * m : nullptr;
#define FK_SPMV(RBV) k_band_spmv<T, RBV><<<nblocks, CG_T, 0, s>>>(band, nb, xb, ub, m, Rb, bo, part, NQ, gb, ctl, R, r0)
        if (Rb <= 1) FK_SPMV(1);
        else if (Rb <= 2) FK_SPMV(2);
        else if (Rb <= 4) FK_SPMV(4);
        else if (Rb <= 8) FK_SPMV(8);
        else if (Rb <= 16) FK_SPMV(16);
        else FK_SPMV(32);
#undef FK_SPMV
        FK_LAUNCH();
    }
    return FKSKI_OK;
}

// ------------------------------------------------------------------ small vector kernels
template <typename T>
__global__ void k_scale(const T *__restrict__ a, T *__restrict__ out, int64_t n, double c) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (T)(c * (double)a[e]);
}

// out[r][i] = x[r][i] + coef[r] * g[r][i] (coef from S field F of R), or + c0 * g when S == null
template <typename T>
__global__ void k_axpy_rhs(const T *__restrict__ x, const T *__restrict__ g, T *__restrict__ out, int64_t m, int R,
                           const double *__restrict__ S, int F, double c0) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / m);
        const double c = S ? S[F * R + r] : c0;
        out[e] = (T)((double)x[e] + c * (double)g[e]);
    }
}

template <typename T>
__global__ void k_convert(const void *__restrict__ in, int in_dbl, T *__restrict__ out, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = in_dbl ? (T)((const double *)in)[e] : (T)((const float *)in)[e];
}

// partial dots for NQ pairs (a_q, b_q) per rhs: part[blk][r][q]
template <typename T, int NQ>
__global__ void __launch_bounds__(CG_T) k_dots(const T *__restrict__ a0, const T *__restrict__ b0, const T *__restrict__ a1,
                                               const T *__restrict__ b1, int64_t m, int R, double *__restrict__ part) {
    __shared__ double sh[CG_T / 32];
    for (int r = 0; r < R; ++r) {
        T acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = T(0);
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
            const int64_t e = (int64_t)r * m + j;
            acc[0] = fma(a0[e], b0[e], acc[0]);
            if (NQ > 1) acc[1] = fma(a1[e], b1[e], acc[1]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double s = block_sum<T>(acc[q], sh);
            if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * R + r * NQ + q] = s;
        }
    }
}

// Plain FP64 sums of partials into out[r*NQ + q] (one warp per (r, q)).
__global__ void k_fin_sums(const double *__restrict__ part, int nparts, int R, int NQ, double *__restrict__ out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= R * NQ) return;
    const double s = warp_sum_partials(part, nparts, R, NQ, w / NQ, w % NQ);
    if ((threadIdx.x & 31) == 0) out[w] = s;
}

// ------------------------------------------------------------------ Alg. 5 kernels
template <typename T>
__global__ void __launch_bounds__(CG_T) k_cg5_xr(int64_t m, int R, T *__restrict__ xd, T *__restrict__ r,
                                                  const T *__restrict__ s, const T *__restrict__ z,
                                                  const double *__restrict__ S, const int *__restrict__ done,
                                                  const CgCtl *__restrict__ ctl) {
    if (ctl->all_done) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(e / m);
        if (done[rr]) continue;
        const T a = (T)S[F_ALPHA * R + rr];
        xd[e] = fma(a, s[e], xd[e]);
        r[e] = fma(-a, z[e], r[e]);
    }
}

// s = u + beta s; z = v + beta z; partial q0 = s.z
template <typename T>
__global__ void __launch_bounds__(CG_T) k_cg5_sz(int64_t m, int R, const T *__restrict__ u, const T *__restrict__ v,
                                                  T *__restrict__ s, T *__restrict__ z, const double *__restrict__ S,
                                                  const int *__restrict__ done, double *__restrict__ part,
                                                  const CgCtl *__restrict__ ctl) {
    if (ctl->all_done) return;
    __shared__ double sh[CG_T / 32];
    for (int r = 0; r < R; ++r) {
        T acc = T(0);
        if (!done[r]) {
            const T b = (T)S[F_BETA * R + r];
            for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
                const int64_t e = (int64_t)r * m + j;
                const T sn = fma(b, s[e], u[e]);
                const T zn = fma(b, z[e], v[e]);
                s[e] = sn;
                z[e] = zn;
                acc = fma(sn, zn, acc);
            }
        }
        const double tot = block_sum<T>(acc, sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * R + r] = tot;
    }
}

// gamma_new = u.r; convergence; beta.  init: first pass (no alpha step taken yet).
__global__ void k_cg5_fin_gamma(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ done,
                                int *__restrict__ iters, double *__restrict__ hist_beta, CgCtl *__restrict__ ctl, int init) {
    if (ctl->all_done) return;
    const int R = ctl->R;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = w; r < R; r += blockDim.x >> 5) {
        const double g = warp_sum_partials(part, nparts, R, 1, r, 0);
        if (lane == 0 && !done[r]) {
            S[F_GNEW * R + r] = g;
            S[F_RES * R + r] = g;
            if (!isfinite(g)) {
                done[r] = 1;
                iters[r] = init ? 0 : ctl->iter + 1;
                atomicOr(&ctl->status, ST_BREAKDOWN);
            } else if (g <= S[F_EPS * R + r]) {
                done[r] = 1;
                iters[r] = init ? 0 : ctl->iter + 1;
            } else if (init) {
                S[F_BETA * R + r] = 0.0;
            } else {
                const double be = g / S[F_GAMMA * R + r];
                S[F_BETA * R + r] = be;
                hist_beta[(int64_t)ctl->iter * R + r] = be;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int r = 0; r < R; ++r) all &= done[r];
        if (all) ctl->all_done = 1;
    }
}

// delta = s.z; alpha = gamma_new / delta; iteration counter.
__global__ void k_cg5_fin_delta(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ done,
                                int *__restrict__ iters, double *__restrict__ hist_alpha, CgCtl *__restrict__ ctl, int init) {
    if (ctl->all_done) return;
    const int R = ctl->R;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = init ? 0 : ctl->iter + 1;
    for (int r = w; r < R; r += blockDim.x >> 5) {
        const double dl = warp_sum_partials(part, nparts, R, 1, r, 0);
        if (lane == 0 && !done[r]) {
            const double gn = S[F_GNEW * R + r];
            S[F_DELTA * R + r] = dl;
            if (!(dl > 0.0) || !isfinite(dl)) {
                done[r] = 1;
                iters[r] = k;
                atomicOr(&ctl->status, ST_BREAKDOWN);
            } else {
                const double a = gn / dl;
                S[F_ALPHA * R + r] = a;
                S[F_GAMMA * R + r] = gn;
                if (k < ctl->maxiter) hist_alpha[(int64_t)k * R + r] = a;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!init) ctl->iter += 1;
        int all = 1;
        for (int r = 0; r < R; ++r) all &= done[r];
        if (ctl->iter >= ctl->maxiter) {
            for (int r = 0; r < R; ++r)
                if (!done[r]) { done[r] = 1; iters[r] = ctl->maxiter; }
            all = 1;
        }
        if (all) ctl->all_done = 1;
    }
}

// ------------------------------------------------------------------ Alg. 3 kernels
// x += a p; xd += a s; r -= a (z + cp kg)
template <typename T>
__global__ void __launch_bounds__(CG_T) k_cg3_xr(int64_t m, int R, T *__restrict__ x, T *__restrict__ xd, T *__restrict__ r,
                                                  const T *__restrict__ p, const T *__restrict__ s, const T *__restrict__ z,
                                                  const T *__restrict__ kg, const double *__restrict__ S,
                                                  const int *__restrict__ done, const CgCtl *__restrict__ ctl) {
    if (ctl->all_done) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(e / m);
        if (done[rr]) continue;
        const T a = (T)S[F_ALPHA * R + rr];
        const T cp = (T)S[F_CP * R + rr];
        x[e] = fma(a, p[e], x[e]);
        xd[e] = fma(a, s[e], xd[e]);
        r[e] = fma(-a, fma(cp, kg[e], z[e]), r[e]);
    }
}

// p = r + beta p; s = u + beta s; z = v + beta z; partial dots s.z, s.kg, p.g, z.g
template <typename T>
__global__ void __launch_bounds__(CG_T) k_cg3_psz(int64_t m, int R, const T *__restrict__ r, const T *__restrict__ u,
                                                   const T *__restrict__ v, T *__restrict__ p, T *__restrict__ s, T *__restrict__ z,
                                                   const T *__restrict__ g, const T *__restrict__ kg,
                                                   const double *__restrict__ S, const int *__restrict__ done,
                                                   double *__restrict__ part, const CgCtl *__restrict__ ctl) {
    if (ctl->all_done) return;
    __shared__ double sh[CG_T / 32];
    for (int rr = 0; rr < R; ++rr) {
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        if (!done[rr]) {
            const T b = (T)S[F_BETA * R + rr];
            for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
                const int64_t e = (int64_t)rr * m + j;
                const T pn = fma(b, p[e], r[e]);
                const T sn = fma(b, s[e], u[e]);
                const T zn = fma(b, z[e], v[e]);
                p[e] = pn;
                s[e] = sn;
                z[e] = zn;
                a0 = fma(sn, zn, a0);
                a1 = fma(sn, kg[e], a1);
                a2 = fma(pn, g[e], a2);
                a3 = fma(zn, g[e], a3);
            }
        }
        const double t0 = block_sum<T>(a0, sh);
        const double t1 = block_sum<T>(a1, sh);
        const double t2 = block_sum<T>(a2, sh);
        const double t3 = block_sum<T>(a3, sh);
        if (threadIdx.x == 0) {
            double *pp = part + (int64_t)blockIdx.x * 4 * R + rr * 4;
            pp[0] = t0; pp[1] = t1; pp[2] = t2; pp[3] = t3;
        }
    }
}

// gamma_new = u.r + 2 cr (r.g) + cr^2 rho0 (Claim 4 with the stored W^T r0 and r0^T r0)
__global__ void k_cg3_fin_gamma(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ done,
                                int *__restrict__ iters, double *__restrict__ hist_beta, CgCtl *__restrict__ ctl) {
    if (ctl->all_done) return;
    const int R = ctl->R;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = w; r < R; r += blockDim.x >> 5) {
        const double ur = warp_sum_partials(part, nparts, R, 2, r, 0);
        const double rg = warp_sum_partials(part, nparts, R, 2, r, 1);
        if (lane == 0 && !done[r]) {
            // the step x += alpha p, r -= alpha A p has just been taken: update the coefficients
            const double a = S[F_ALPHA * R + r], cp0 = S[F_CP * R + r];
            S[F_CX * R + r] += a * cp0;
            const double cr = S[F_CR * R + r] - a * ctl->sig2 * cp0;
            S[F_CR * R + r] = cr;
            const double g = ur + 2.0 * cr * rg + cr * cr * S[F_RHO0 * R + r];
            S[F_GNEW * R + r] = g;
            S[F_RES * R + r] = g;
            if (!isfinite(g)) {
                done[r] = 1;
                iters[r] = ctl->iter + 1;
                atomicOr(&ctl->status, ST_BREAKDOWN);
            } else if (g <= S[F_EPS * R + r]) {
                done[r] = 1;
                iters[r] = ctl->iter + 1;
            } else {
                const double be = g / S[F_GAMMA * R + r];
                S[F_BETA * R + r] = be;
                hist_beta[(int64_t)ctl->iter * R + r] = be;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int r = 0; r < R; ++r) all &= done[r];
        if (all) ctl->all_done = 1;
    }
}

// cp' = cr + beta cp; denom = <p, A p> (Claim 4); alpha for the next step.
__global__ void k_cg3_fin_delta(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ done,
                                int *__restrict__ iters, double *__restrict__ hist_alpha, CgCtl *__restrict__ ctl) {
    if (ctl->all_done) return;
    const int R = ctl->R;
    const double s2 = ctl->sig2;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = ctl->iter + 1;
    for (int r = w; r < R; r += blockDim.x >> 5) {
        const double sz = warp_sum_partials(part, nparts, R, 4, r, 0);
        const double skg = warp_sum_partials(part, nparts, R, 4, r, 1);
        const double pg = warp_sum_partials(part, nparts, R, 4, r, 2);
        const double zg = warp_sum_partials(part, nparts, R, 4, r, 3);
        if (lane == 0 && !done[r]) {
            const double cp = S[F_CR * R + r] + S[F_BETA * R + r] * S[F_CP * R + r];
            const double cq = s2 * cp;
            const double den = sz + cp * skg + cq * pg + cp * zg + cp * cp * S[F_GKG * R + r] + cp * cq * S[F_RHO0 * R + r];
            if (!(den > 0.0) || !isfinite(den)) {
                done[r] = 1;
                iters[r] = k;
                atomicOr(&ctl->status, ST_BREAKDOWN);
            } else {
                const double gn = S[F_GNEW * R + r];
                const double a = gn / den;
                S[F_CP * R + r] = cp;
                S[F_ALPHA * R + r] = a;
                S[F_GAMMA * R + r] = gn;
                if (k < ctl->maxiter) hist_alpha[(int64_t)k * R + r] = a;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->iter += 1;
        int all = 1;
        for (int r = 0; r < R; ++r) all &= done[r];
        if (ctl->iter >= ctl->maxiter) {
            for (int r = 0; r < R; ++r)
                if (!done[r]) { done[r] = 1; iters[r] = ctl->maxiter; }
            all = 1;
        }
        if (all) ctl->all_done = 1;
    }
}

// Alg. 3 start: x0 = 0, r0 = b: cr = cp = 1, cx = 0, gamma = rho0, alpha_0 = rho0 / (g.Kg + s2 rho0).
__global__ void k_cg3_init(double *__restrict__ S, const double *__restrict__ gkg, int *__restrict__ done,
                           int *__restrict__ iters, double *__restrict__ hist_alpha, CgCtl *__restrict__ ctl) {
    const int R = ctl->R;
    const double s2 = ctl->sig2;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const double rho0 = S[F_RHO0 * R + r];
        const double den = gkg[r] + s2 * rho0;
        S[F_GKG * R + r] = gkg[r];
        S[F_GAMMA * R + r] = rho0;
        S[F_RES * R + r] = rho0;
        S[F_CP * R + r] = 1.0;
        done[r] = 0;
        iters[r] = 0;
        if (rho0 <= S[F_EPS * R + r]) {
            done[r] = 1;
            continue;
        }
        if (!(den > 0.0) || !isfinite(den)) {
            done[r] = 1;
            atomicOr(&ctl->status, ST_BREAKDOWN);
            continue;
        }
        const double a = rho0 / den;
        S[F_ALPHA * R + r] = a;
        S[F_CX * R + r] = 0.0;
        S[F_CR * R + r] = 1.0;
        hist_alpha[r] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int r = 0; r < R; ++r) all &= done[r];
        ctl->all_done = all;
    }
}

// ------------------------------------------------------------------ workspace
struct SolveWork {
    KgOp *kg[2];
    void *buf;
    size_t buf_bytes;
    double *S;
    double *part;
    int *done;
    int *iters;
    CgCtl *ctl;
    double *hist;     // alpha then beta, maxiter x R each
    size_t hist_cap;  // entries per array
    int *hflag;       // pinned host: all_done
    cudaStream_t ws;  // internal stream for graph capture (the caller's may be the legacy stream)
    cudaEvent_t ev;
    // stored solutions for the log-likelihood backward pass
    void *sol;
    size_t sol_bytes;
    int sol_valid;
    int sol_dtype;
    double sol_sig2, sol_ell[3], sol_s;
    int sol_type;
};

void free_solve_work(SolveWork *w) {
    if (!w) return;
    for (int i = 0; i < 2; ++i) kgop_destroy(w->kg[i]);
    if (w->buf) cudaFree(w->buf);
    if (w->S) cudaFree(w->S);
    if (w->part) cudaFree(w->part);
    if (w->done) cudaFree(w->done);
    if (w->iters) cudaFree(w->iters);
    if (w->ctl) cudaFree(w->ctl);
    if (w->hist) cudaFree(w->hist);
    if (w->hflag) cudaFreeHost(w->hflag);
    if (w->ws) cudaStreamDestroy(w->ws);
    if (w->ev) cudaEventDestroy(w->ev);
    if (w->sol) cudaFree(w->sol);
    delete w;
}

static int dev_alloc(void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return FKSKI_E_OOM;
    }
    return FKSKI_OK;
}

constexpr int MAX_R = kMaxProbes + 1;
constexpr int NPART = 152 * 4;

static int work_get(fkski_stats *st, SolveWork **out) {
    if (!st->work) {
        SolveWork *w = new SolveWork;
        memset(w, 0, sizeof(*w));
        st->work = w;
        FK_TRY(dev_alloc((void **)&w->S, sizeof(double) * (NF * MAX_R + MAX_R + 8)));
        FK_TRY(dev_alloc((void **)&w->part, sizeof(double) * NPART * 4 * MAX_R));
        FK_TRY(dev_alloc((void **)&w->done, sizeof(int) * MAX_R));
        FK_TRY(dev_alloc((void **)&w->iters, sizeof(int) * MAX_R));
        FK_TRY(dev_alloc((void **)&w->ctl, sizeof(CgCtl)));
        if (cudaMallocHost((void **)&w->hflag, sizeof(int) * 4) != cudaSuccess) {
            cudaGetLastError();
            return FKSKI_E_OOM;
        }
        FK_CUDA(cudaStreamCreateWithFlags(&w->ws, cudaStreamNonBlocking));
        FK_CUDA(cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming));
    }
    *out = st->work;
    return FKSKI_OK;
}

static int work_kg(fkski_stats *st, SolveWork *w, int dtype, KgOp **op) {
    const int i = dtype == FKSKI_F32 ? 0 : 1;
    if (!w->kg[i]) FK_TRY(kgop_create(&st->grid, dtype, &w->kg[i]));
    *op = w->kg[i];
    return FKSKI_OK;
}

static int work_buf(SolveWork *w, size_t bytes) {
    if (w->buf_bytes >= bytes) return FKSKI_OK;
    if (w->buf) cudaFree(w->buf);
    w->buf = nullptr;
    w->buf_bytes = 0;
    FK_TRY(dev_alloc(&w->buf, bytes));
    w->buf_bytes = bytes;
    return FKSKI_OK;
}

static int work_hist(SolveWork *w, int R, int maxiter) {
    const size_t need = (size_t)R * (size_t)(maxiter + 1);
    if (w->hist_cap >= need) return FKSKI_OK;
    if (w->hist) cudaFree(w->hist);
    w->hist = nullptr;
    w->hist_cap = 0;
    FK_TRY(dev_alloc((void **)&w->hist, sizeof(double) * 2 * need));
    w->hist_cap = need;
    return FKSKI_OK;
}

// Converted copies of the statistics in the solve precision.
template <typename T>
static int stats_as(fkski_stats *st, const T **band, const T **wty, const T **wtz, cudaStream_t s) {
    const int want = sizeof(T) == 4 ? FKSKI_F32 : FKSKI_F64;
    const int64_t nb = ipow(7, st->d) * st->m;
    if (st->dtype == want) {
        *band = (const T *)st->band;
        *wty = (const T *)st->wty;
        *wtz = (const T *)st->wtz;
        return FKSKI_OK;
    }
    if (!st->band_alt) {
        FK_TRY(dev_alloc(&st->band_alt, sizeof(T) * nb));
        FK_TRY(dev_alloc(&st->wty_alt, sizeof(T) * st->m));
        const unsigned g = (unsigned)std::min<int64_t>(cdiv(nb, 256), 4096);
        k_convert<T><<<g, 256, 0, s>>>(st->band, st->dtype == FKSKI_F64, (T *)st->band_alt, nb);
        FK_LAUNCH();
        k_convert<T><<<256, 256, 0, s>>>(st->wty, st->dtype == FKSKI_F64, (T *)st->wty_alt, st->m);
        FK_LAUNCH();
        if (st->nprobes > 0) {
            FK_TRY(dev_alloc(&st->wtz_alt, sizeof(T) * st->nprobes * st->m));
            k_convert<T><<<1024, 256, 0, s>>>(st->wtz, st->dtype == FKSKI_F64, (T *)st->wtz_alt, st->nprobes * st->m);
            FK_LAUNCH();
        }
    }
    *band = (const T *)st->band_alt;
    *wty = (const T *)st->wty_alt;
    *wtz = (const T *)st->wtz_alt;
    return FKSKI_OK;
}

int stats_band_as(fkski_stats *st, int dtype, const void **band, const void **wty, const void **wtz, cudaStream_t s) {
    if (dtype == FKSKI_F32) return stats_as<float>(st, (const float **)band, (const float **)wty, (const float **)wtz, s);
    return stats_as<double>(st, (const double **)band, (const double **)wty, (const double **)wtz, s);
}

// Run the captured iteration body (captured on w->ws) until convergence or maxiter; the
// internal stream first waits for the caller's stream, and the caller's stream waits for it.
static int run_graph_loop(cudaGraphExec_t exec, SolveWork *w, int maxiter, int check, cudaStream_t s) {
    FK_CUDA(cudaEventRecord(w->ev, s));
    FK_CUDA(cudaStreamWaitEvent(w->ws, w->ev, 0));
    int done_iters = 0;
    while (done_iters < maxiter + check) {
        FK_CUDA(cudaGraphLaunch(exec, w->ws));
        done_iters += check;
        FK_CUDA(cudaMemcpyAsync(w->hflag, &w->ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, w->ws));
        FK_CUDA(cudaStreamSynchronize(w->ws));
        if (w->hflag[0]) break;
    }
    FK_CUDA(cudaEventRecord(w->ev, w->ws));
    FK_CUDA(cudaStreamWaitEvent(s, w->ev, 0));
    return FKSKI_OK;
}

template <typename T>
struct Alg3Vecs {
    T *r, *p, *x, *xd, *u, *v, *s, *z, *g, *kg;
};

// ------------------------------------------------------------------ Alg. 5 solve
template <typename T>
static int solve_alg5(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, T *a_out, T *v_out,
                      fkski_info *info, cudaStream_t s) {
    SolveWork *w;
    FK_TRY(work_get(st, &w));
    const int dt = sizeof(T) == 4 ? FKSKI_F32 : FKSKI_F64;
    KgOp *kg;
    FK_TRY(work_kg(st, w, dt, &kg));
    FK_TRY(kgop_set(kg, kern, -1, s));
    const T *band, *wty, *wtz;
    FK_TRY(stats_as<T>(st, &band, &wty, &wtz, s));
    const int64_t m = st->m;
    const int R = 1;
    FK_TRY(work_buf(w, sizeof(T) * 6 * m));
    T *r = (T *)w->buf, *u = r + m, *v = u + m, *sv = v + m, *z = sv + m, *xd = z + m;
    FK_TRY(work_hist(w, R, o->maxiter));
    double *ha = w->hist, *hb = w->hist + w->hist_cap;
    const double s2 = kern->noise_var;
    // scalars
    CgCtl hc;
    memset(&hc, 0, sizeof(hc));
    hc.maxiter = o->maxiter;
    hc.R = R;
    hc.sig2 = s2;
    FK_CUDA(cudaMemcpyAsync(w->ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, s));
    double hS[NF];
    memset(hS, 0, sizeof(hS));
    hS[F_EPS] = o->rtol * o->rtol * st->yty;
    hS[F_RHO0] = st->yty;
    FK_CUDA(cudaMemcpyAsync(w->S, hS, sizeof(hS), cudaMemcpyHostToDevice, s));
    FK_CUDA(cudaMemsetAsync(w->done, 0, sizeof(int) * R, s));
    FK_CUDA(cudaMemsetAsync(w->iters, 0, sizeof(int) * R, s));
    FK_CUDA(cudaMemsetAsync(sv, 0, sizeof(T) * 2 * m, s));  // s, z
    FK_CUDA(cudaMemsetAsync(xd, 0, sizeof(T) * m, s));
    // r0_hat = -K_G W^T y / sigma^2
    FK_TRY(kgop_apply(kg, wty, u, 1, nullptr, 0.0, s));
    const unsigned gb = (unsigned)grid_blocks(m);
    k_scale<T><<<gb, CG_T, 0, s>>>(u, r, m, -1.0 / s2);
    FK_LAUNCH();
    const double *sig2_dev = &w->ctl->sig2;
    // init pass: B(r0), gamma0, s0 = u0, z0 = v0, delta0, alpha0
    FK_TRY(launch_spmv<T>(band, st->grid, r, u, m, R, w->part, 1, nullptr, w->ctl, gb, s));
    k_cg5_fin_gamma<<<1, 256, 0, s>>>(w->part, gb, w->S, w->done, w->iters, hb, w->ctl, 1);
    FK_LAUNCH();
    FK_TRY(kgop_apply_dev(kg, u, v, 1, r, sig2_dev, s));
    k_cg5_sz<T><<<gb, CG_T, 0, s>>>(m, R, u, v, sv, z, w->S, w->done, w->part, w->ctl);
    FK_LAUNCH();
    k_cg5_fin_delta<<<1, 256, 0, s>>>(w->part, gb, w->S, w->done, w->iters, ha, w->ctl, 1);
    FK_LAUNCH();
    // capture `check` iterations
    const int check = std::max(1, o->check_every);
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    const cudaStream_t cs = w->ws;
    FK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    int rc = FKSKI_OK;
    for (int it = 0; it < check && rc == FKSKI_OK; ++it) {
        k_cg5_xr<T><<<gb, CG_T, 0, cs>>>(m, R, xd, r, sv, z, w->S, w->done, w->ctl);
        rc = launch_spmv<T>(band, st->grid, r, u, m, R, w->part, 1, nullptr, w->ctl, gb, cs);
        if (rc) break;
        k_cg5_fin_gamma<<<1, 256, 0, cs>>>(w->part, gb, w->S, w->done, w->iters, hb, w->ctl, 0);
        rc = kgop_apply_dev(kg, u, v, 1, r, sig2_dev, cs);
        if (rc) break;
        k_cg5_sz<T><<<gb, CG_T, 0, cs>>>(m, R, u, v, sv, z, w->S, w->done, w->part, w->ctl);
        k_cg5_fin_delta<<<1, 256, 0, cs>>>(w->part, gb, w->S, w->done, w->iters, ha, w->ctl, 0);
    }
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (rc != FKSKI_OK) return rc;
    FK_CUDA(ce);
    FK_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    rc = run_graph_loop(exec, w, o->maxiter, check, s);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (rc) return rc;
    // a = xd + W^T y / sigma^2 ; v = K a
    k_axpy_rhs<T><<<gb, CG_T, 0, s>>>(xd, wty, a_out, m, 1, nullptr, 0, 1.0 / s2);
    FK_LAUNCH();
    FK_TRY(kgop_apply(kg, a_out, v_out, 1, nullptr, 0.0, s));
    // report
    CgCtl hc2;
    int hit = 0;
    double hS2[NF * 1];
    FK_CUDA(cudaMemcpyAsync(&hc2, w->ctl, sizeof(hc2), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaMemcpyAsync(&hit, w->iters, sizeof(int), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaMemcpyAsync(hS2, w->S, sizeof(hS2), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaStreamSynchronize(s));
    const double res = std::sqrt(std::max(hS2[F_RES], 0.0) / std::max(st->yty, 1e-300));
    int status = FKSKI_OK;
    if (hc2.status & ST_BREAKDOWN) status = FKSKI_E_BREAKDOWN;
    else if (hS2[F_RES] > hS2[F_EPS]) status = FKSKI_E_NOT_CONVERGED;
    if (info) {
        info->iters = hit;
        info->iters_rhs[0] = hit;
        info->rel_residual = res;
        info->status = status;
    }
    return status;
}

// ------------------------------------------------------------------ Alg. 3 batched solve
// Right-hand sides: b_0 = y (g = W^T y, rho0 = y^T y) and b_p = z_p (g = W^T z_p, rho0 = z_p^T z_p).
// Leaves the compressed solutions in the work buffer (see Alg3Vecs) and the CG coefficients in
// the history arrays.
template <typename T>
int solve_alg3_batched(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, int R, Alg3Vecs<T> &V,
                       int *iters_host, double *res_host, int *status_out, cudaStream_t s) {
    SolveWork *w;
    FK_TRY(work_get(st, &w));
    const int dt = sizeof(T) == 4 ? FKSKI_F32 : FKSKI_F64;
    KgOp *kg;
    FK_TRY(work_kg(st, w, dt, &kg));
    FK_TRY(kgop_set(kg, kern, -1, s));
    const T *band, *wty, *wtz;
    FK_TRY(stats_as<T>(st, &band, &wty, &wtz, s));
    const int64_t m = st->m;
    FK_TRY(work_buf(w, sizeof(T) * 10 * (size_t)R * m));
    T *b = (T *)w->buf;
    V.r = b; V.p = b + R * m; V.x = b + 2 * R * m; V.xd = b + 3 * R * m; V.u = b + 4 * R * m;
    V.v = b + 5 * R * m; V.s = b + 6 * R * m; V.z = b + 7 * R * m; V.g = b + 8 * R * m; V.kg = b + 9 * R * m;
    FK_TRY(work_hist(w, R, o->maxiter));
    double *ha = w->hist, *hb = w->hist + w->hist_cap;
    const double s2 = kern->noise_var;
    // g = [W^T y, W^T z_1..]
    FK_CUDA(cudaMemcpyAsync(V.g, wty, sizeof(T) * m, cudaMemcpyDeviceToDevice, s));
    if (R > 1) FK_CUDA(cudaMemcpyAsync(V.g + m, wtz, sizeof(T) * (R - 1) * m, cudaMemcpyDeviceToDevice, s));
    FK_CUDA(cudaMemsetAsync(b, 0, sizeof(T) * 8 * (size_t)R * m, s));
    FK_TRY(kgop_apply(kg, V.g, V.kg, R, nullptr, 0.0, s));
    CgCtl hc;
    memset(&hc, 0, sizeof(hc));
    hc.maxiter = o->maxiter;
    hc.R = R;
    hc.sig2 = s2;
    FK_CUDA(cudaMemcpyAsync(w->ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, s));
    std::vector<double> hS((size_t)NF * R, 0.0);
    for (int r = 0; r < R; ++r) {
        const double rho = r == 0 ? st->yty : st->ztz[r - 1];
        hS[F_RHO0 * R + r] = rho;
        hS[F_EPS * R + r] = o->rtol * o->rtol * rho;
    }
    FK_CUDA(cudaMemcpyAsync(w->S, hS.data(), sizeof(double) * NF * R, cudaMemcpyHostToDevice, s));
    const unsigned gb = (unsigned)grid_blocks(m);
    double *gkg = w->S + NF * MAX_R;  // scratch after the fields
    k_dots<T, 1><<<gb, CG_T, 0, s>>>(V.g, V.kg, nullptr, nullptr, m, R, w->part);
    FK_LAUNCH();
    // reuse w->part tail for the sums
    k_fin_sums<<<(unsigned)cdiv(R * 32, 256), 256, 0, s>>>(w->part, gb, R, 1, gkg);
    FK_LAUNCH();
    k_cg3_init<<<1, 256, 0, s>>>(w->S, gkg, w->done, w->iters, ha, w->ctl);
    FK_LAUNCH();
    const double *sig2_dev = &w->ctl->sig2;
    const int check = std::max(1, o->check_every);
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    const cudaStream_t cs = w->ws;
    FK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    int rc = FKSKI_OK;
    for (int it = 0; it < check && rc == FKSKI_OK; ++it) {
        k_cg3_xr<T><<<gb, CG_T, 0, cs>>>(m, R, V.x, V.xd, V.r, V.p, V.s, V.z, V.kg, w->S, w->done, w->ctl);
        rc = launch_spmv<T>(band, st->grid, V.r, V.u, m, R, w->part, 2, V.g, w->ctl, gb, cs);
        if (rc) break;
        k_cg3_fin_gamma<<<1, 256, 0, cs>>>(w->part, gb, w->S, w->done, w->iters, hb, w->ctl);
        rc = kgop_apply_dev(kg, V.u, V.v, R, V.r, sig2_dev, cs);
        if (rc) break;
        k_cg3_psz<T><<<gb, CG_T, 0, cs>>>(m, R, V.r, V.u, V.v, V.p, V.s, V.z, V.g, V.kg, w->S, w->done, w->part, w->ctl);
        k_cg3_fin_delta<<<1, 256, 0, cs>>>(w->part, gb, w->S, w->done, w->iters, ha, w->ctl);
    }
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (rc != FKSKI_OK) return rc;
    FK_CUDA(ce);
    FK_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    rc = run_graph_loop(exec, w, o->maxiter, check, s);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (rc) return rc;
    CgCtl hc2;
    std::vector<double> hS2((size_t)NF * R);
    FK_CUDA(cudaMemcpyAsync(&hc2, w->ctl, sizeof(hc2), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaMemcpyAsync(iters_host, w->iters, sizeof(int) * R, cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaMemcpyAsync(hS2.data(), w->S, sizeof(double) * NF * R, cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaStreamSynchronize(s));
    int status = FKSKI_OK;
    for (int r = 0; r < R; ++r) {
        res_host[r] = std::sqrt(std::max(hS2[F_RES * R + r], 0.0) / std::max(hS2[F_RHO0 * R + r], 1e-300));
        if (hS2[F_RES * R + r] > hS2[F_EPS * R + r] && status == FKSKI_OK) status = FKSKI_E_NOT_CONVERGED;
    }
    if (hc2.status & ST_BREAKDOWN) status = FKSKI_E_BREAKDOWN;
    *status_out = status;
    return FKSKI_OK;
}

template int solve_alg3_batched<float>(fkski_stats *, const fkski_kernel *, const fkski_opts *, int, Alg3Vecs<float> &,
                                       int *, double *, int *, cudaStream_t);
template int solve_alg3_batched<double>(fkski_stats *, const fkski_kernel *, const fkski_opts *, int, Alg3Vecs<double> &,
                                        int *, double *, int *, cudaStream_t);

template <typename T>
static int solve_alg3_mean(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, T *a_out, T *v_out,
                           fkski_info *info, cudaStream_t s) {
    Alg3Vecs<T> V;
    int it = 0, status = 0;
    double res = 0.0;
    FK_TRY(solve_alg3_batched<T>(st, kern, o, 1, V, &it, &res, &status, s));
    SolveWork *w = st->work;
    const int64_t m = st->m;
    const unsigned gb = (unsigned)grid_blocks(m);
    // W^T x = xd + cx W^T y
    k_axpy_rhs<T><<<gb, CG_T, 0, s>>>(V.xd, V.g, a_out, m, 1, w->S, F_CX, 0.0);
    FK_LAUNCH();
    KgOp *kg = w->kg[sizeof(T) == 4 ? 0 : 1];
    FK_TRY(kgop_apply(kg, a_out, v_out, 1, nullptr, 0.0, s));
    FK_CUDA(cudaStreamSynchronize(s));
    if (info) {
        info->iters = it;
        info->iters_rhs[0] = it;
        info->rel_residual = res;
        info->status = status;
    }
    return status;
}

int solve_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, void *a_out, void *v_out,
               fkski_info *info, cudaStream_t s) {
    if (!st || !kern || !a_out || !v_out) return FKSKI_E_INVALID_ARG;
    fkski_opts o;
    if (opts) o = *opts; else fkski_default_opts(&o);
    if (!(kern->noise_var > 0.0) || !std::isfinite(kern->noise_var)) return FKSKI_E_INVALID_ARG;
    if (o.maxiter < 1 || !(o.rtol >= 0.0)) return FKSKI_E_INVALID_ARG;
    if (info) memset(info, 0, sizeof(*info));
    const bool dbl = o.precision == FKSKI_DOUBLE;
    if (o.x0_mode == FKSKI_X0_Y_OVER_S2) {
        return dbl ? solve_alg5<double>(st, kern, &o, (double *)a_out, (double *)v_out, info, s)
                   : solve_alg5<float>(st, kern, &o, (float *)a_out, (float *)v_out, info, s);
    }
    if (o.x0_mode != FKSKI_X0_ZERO) return FKSKI_E_INVALID_ARG;
    return dbl ? solve_alg3_mean<double>(st, kern, &o, (double *)a_out, (double *)v_out, info, s)
               : solve_alg3_mean<float>(st, kern, &o, (float *)a_out, (float *)v_out, info, s);
}

int band_mvm_impl(const fkski_stats *stc, const void *x, void *u, int nrhs, int dtype, cudaStream_t s) {
    if (!stc || !x || !u || nrhs < 1) return FKSKI_E_INVALID_ARG;
    fkski_stats *st = const_cast<fkski_stats *>(stc);
    const unsigned gb = (unsigned)grid_blocks(st->m);
    if (dtype == FKSKI_F32) {
        const float *band, *wty, *wtz;
        FK_TRY(stats_as<float>(st, &band, &wty, &wtz, s));
        return launch_spmv<float>(band, st->grid, (const float *)x, (float *)u, st->m, nrhs, nullptr, 1, nullptr,
                                  nullptr, gb, s);
    }
    if (dtype != FKSKI_F64) return FKSKI_E_INVALID_ARG;
    const double *band, *wty, *wtz;
    FK_TRY(stats_as<double>(st, &band, &wty, &wtz, s));
    return launch_spmv<double>(band, st->grid, (const double *)x, (double *)u, st->m, nrhs, nullptr, 1, nullptr,
                               nullptr, gb, s);
}

// exported for grad.cu
int alg3_for_grad_f32(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, int R, Alg3Vecs<float> &V,
                      int *iters, double *res, int *status, cudaStream_t s) {
    return solve_alg3_batched<float>(st, kern, o, R, V, iters, res, status, s);
}
int alg3_for_grad_f64(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, int R, Alg3Vecs<double> &V,
                      int *iters, double *res, int *status, cudaStream_t s) {
    return solve_alg3_batched<double>(st, kern, o, R, V, iters, res, status, s);
}

// ------------------------------------------------------------------ predict
// mu(x*) = sum over the 4^d stencil nodes of w(x*) v  (Def. 1 / Fact 2 mean)
template <typename TX, typename TV, int D>
__global__ void k_predict(const TX *__restrict__ Xs, int64_t ns, KeyParams kp, const TV *__restrict__ v,
                          TV *__restrict__ mu, int *__restrict__ status, int64_t s1, int64_t s2) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
        int c[3] = {1, 1, 1};
        TX t[3] = {TX(0), TX(0), TX(0)};
        int st = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) st |= axis_cell<TX>(Xs[(int64_t)k * ns + i], kp, k, c[k], t[k]);
        if (st) {
            bad |= (st & 2) ? ST_NONFINITE : ST_OUT_OF_GRID;
            mu[i] = TV(0);
            continue;
        }
        TV w[3][4];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            TX wx[4];
            keys_weights<TX>(t[k], wx);
#pragma unroll
            for (int a = 0; a < 4; ++a) w[k][a] = (TV)wx[a];
        }
        TV acc = TV(0);
        if (D == 1) {
#pragma unroll
            for (int a = 0; a < 4; ++a) acc = fma(w[0][a], v[c[0] - 1 + a], acc);
        } else if (D == 2) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                TV rowacc = TV(0);
                const int64_t base = (int64_t)(c[0] - 1 + a) * s1 + (c[1] - 1);
#pragma unroll
                for (int b = 0; b < 4; ++b) rowacc = fma(w[1][b], v[base + b], rowacc);
                acc = fma(w[0][a], rowacc, acc);
            }
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                TV pl = TV(0);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int64_t base = (int64_t)(c[0] - 1 + a) * s1 + (int64_t)(c[1] - 1 + b) * s2 + (c[2] - 1);
                    TV rowacc = TV(0);
#pragma unroll
                    for (int e = 0; e < 4; ++e) rowacc = fma(w[2][e], v[base + e], rowacc);
                    pl = fma(w[1][b], rowacc, pl);
                }
                acc = fma(w[0][a], pl, acc);
            }
        }
        mu[i] = acc;
    }
    if (bad) atomicOr(status, bad);
}

template <typename TX, typename TV>
static int predict_typed(const fkski_stats *st, const TV *v, const TX *Xs, int64_t ns, TV *mu, cudaStream_t s) {
    const KeyParams kp = make_key_params(st->grid);
    int *dst;
    FK_CUDA(cudaMallocAsync((void **)&dst, sizeof(int), s));
    FK_CUDA(cudaMemsetAsync(dst, 0, sizeof(int), s));
    const int64_t M1 = st->grid.M[1], M2 = st->grid.M[2];
    const int64_t s1 = st->d == 2 ? M1 : M1 * M2, s2 = M2;
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(ns, 256), 152 * 16));
    if (st->d == 1) k_predict<TX, TV, 1><<<gb, 256, 0, s>>>(Xs, ns, kp, v, mu, dst, s1, s2);
    else if (st->d == 2) k_predict<TX, TV, 2><<<gb, 256, 0, s>>>(Xs, ns, kp, v, mu, dst, s1, s2);
    else k_predict<TX, TV, 3><<<gb, 256, 0, s>>>(Xs, ns, kp, v, mu, dst, s1, s2);
    FK_LAUNCH();
    int h = 0;
    FK_CUDA(cudaMemcpyAsync(&h, dst, sizeof(int), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaFreeAsync(dst, s));
    FK_CUDA(cudaStreamSynchronize(s));
    return status_from_bits(h);
}

int predict_impl(const fkski_stats *st, const void *v, int vdtype, const void *Xs, int xdtype, int64_t ns, void *mu,
                 cudaStream_t s) {
    if (!st || !v || !Xs || !mu || ns < 0) return FKSKI_E_INVALID_ARG;
    if (ns == 0) return FKSKI_OK;
    if (vdtype == FKSKI_F32 && xdtype == FKSKI_F32)
        return predict_typed<float, float>(st, (const float *)v, (const float *)Xs, ns, (float *)mu, s);
    if (vdtype == FKSKI_F64 && xdtype == FKSKI_F32)
        return predict_typed<float, double>(st, (const double *)v, (const float *)Xs, ns, (double *)mu, s);
    if (vdtype == FKSKI_F32 && xdtype == FKSKI_F64)
        return predict_typed<double, float>(st, (const float *)v, (const double *)Xs, ns, (float *)mu, s);
    if (vdtype == FKSKI_F64 && xdtype == FKSKI_F64)
        return predict_typed<double, double>(st, (const double *)v, (const double *)Xs, ns, (double *)mu, s);
    return FKSKI_E_INVALID_ARG;
}

}  // namespace fk

namespace fk {
// ------------------------------------------------------------------ hooks for grad.cu
struct GradView {
    double *S;
    double *hist_a;
    double *hist_b;
    int *iters;
    KgOp *kg;
};

int grad_view(fkski_stats *st, int dtype, GradView *gv) {
    SolveWork *w;
    FK_TRY(work_get(st, &w));
    KgOp *kg;
    FK_TRY(work_kg(st, w, dtype, &kg));
    gv->S = w->S;
    gv->hist_a = w->hist;
    gv->hist_b = w->hist + w->hist_cap;
    gv->iters = w->iters;
    gv->kg = kg;
    return FKSKI_OK;
}

int grad_sol_buffer(fkski_stats *st, size_t bytes, void **p) {
    SolveWork *w;
    FK_TRY(work_get(st, &w));
    if (w->sol_bytes < bytes || !w->sol) {
        if (w->sol) cudaFree(w->sol);
        w->sol = nullptr;
        w->sol_bytes = 0;
        w->sol_valid = 0;
        FK_TRY(dev_alloc(&w->sol, std::max<size_t>(bytes, 16)));
        w->sol_bytes = std::max<size_t>(bytes, 16);
    }
    *p = w->sol;
    return FKSKI_OK;
}

void grad_sol_mark(fkski_stats *st, int valid, const fkski_kernel *kern, int dtype) {
    SolveWork *w = st->work;
    if (!w) return;
    w->sol_valid = valid;
    if (!valid) {
        // over the iterate budget: release the solutions, the backward pass recomputes them
        cudaFree(w->sol);
        w->sol = nullptr;
        w->sol_bytes = 0;
        return;
    }
    w->sol_dtype = dtype;
    w->sol_type = kern->type;
    w->sol_sig2 = kern->noise_var;
    w->sol_s = kern->outputscale;
    for (int k = 0; k < 3; ++k) w->sol_ell[k] = kern->lengthscale[k];
}

int grad_sol_valid(fkski_stats *st, const fkski_kernel *kern, int dtype) {
    SolveWork *w = st->work;
    if (!w || !w->sol_valid || !w->sol) return 0;
    if (w->sol_dtype != dtype || w->sol_type != kern->type || w->sol_sig2 != kern->noise_var ||
        w->sol_s != kern->outputscale)
        return 0;
    for (int k = 0; k < st->d; ++k)
        if (w->sol_ell[k] != kern->lengthscale[k]) return 0;
    return 1;
}

int spmv_for_grad(fkski_stats *st, const void *x, void *u, int R, int dtype, cudaStream_t s) {
    return band_mvm_impl(st, x, u, R, dtype, s);
}
}  // namespace fk
