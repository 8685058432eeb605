// m-space solves from the sufficient statistics (Sec. 4, App. B) and posterior-mean prediction.
//
// B(x) = [(K_G W^T W + sigma^2 I) x, W^T W x] is one banded SpMV (Claim 2, 7^d diagonals) feeding
// one K_G application (kg.cu).  One factorized-CG engine runs both variants of App. B:
//   Alg. 5 (simplified EFCG): x0 = y / sigma^2 puts r0 in span(W); iterates r = W r_hat.
//   Alg. 3 (EFCG, x0 = 0):     r = W r_hat + c^r r0, p = W p_hat + c^p r0, x = W x_hat + c^x r0,
//     with the inner products of Claim 4 from the stored W^T r0 and r0^T r0; batched over
//     right-hand sides [y, z_1..z_T] so every B(x) reads the band once.
// Each iteration applies B once (to r_hat) and carries A p through the recurrences of the
// paper's EFCG (z_hat, s_hat).
//
// Precision.  DOUBLE runs the paper's EFCG in FP64 exactly, testing the recursive residual.
// MIXED keeps the Krylov recurrences (r, p, u, v, s, z) in FP32 and the solution x_hat in FP64,
// with "reliable updates": at the end of a captured chunk of `check_every` iterations, every
// right-hand side whose recursive residual fell below delta^2 = 0.01 times its value at the last
// replacement (or below the tolerance) gets its residual replaced by the true one,
//   r_hat = r_hat_0 - (K W^T W + sigma^2 I) x_hat              (Alg. 5)
//   r_hat = -((K W^T W + sigma^2 I) x_hat + c^x K W^T r0)      (Alg. 3),
// computed with an FP64 SpMV and an FP64 K_G; convergence is declared only on that true
// residual.  Without this the FP32 recurrences for A p drift (GP systems have condition numbers
// ~1e6) and the recursive residual detaches from the true one.  Inner products are FP32 within a
// warp (MIXED) and FP64 across warps and blocks, in a fixed order (deterministic).  All scalars
// live in device memory; iterations run as captured CUDA graphs with flags read between launches.
#include "fkski_internal.cuh"

#include <algorithm>
#include <type_traits>
#include <vector>

namespace fk {

constexpr int CG_T = 256;

// per-rhs scalar fields (double S[F * R + r])
enum {
    F_GAMMA = 0, F_GNEW, F_ALPHA, F_BETA, F_CR, F_CP, F_CX, F_RHO0, F_EPS, F_GKG, F_DELTA, F_RES, F_GLAST,
    F_RHOP,  // ||b'||^2 of the compressed base vector b' (GEN)
    F_C0,    // x0 = c0 b (1/sigma^2 for the y / sigma^2 start, else 0)
    F_BG,    // b_hat . W^T b' (GEN, for b^T x)
    NF
};

// per-rhs state: 0 active, 1 converged on the recursive residual (to confirm), 2 finished
enum { RS_ACTIVE = 0, RS_TENTATIVE = 1, RS_FINAL = 2 };

struct CgCtl {
    int iter;      // completed alpha steps
    int all_done;  // every rhs tentative or final: iteration kernels idle
    int all_conf;  // every rhs final: the host stops
    int any_rep;   // some rhs asks for a residual replacement (read by the host after a chunk)
    int status;    // ST_* bits
    int maxiter;
    int R;
    int replace;   // MIXED: reliable updates on; DOUBLE: off
    double sig2;
    double delta2; // replacement trigger: gamma < delta2 * gamma at the last replacement
    unsigned int fin_cnt[2];  // blocks done in the launch whose last block finalises (gamma, delta)
};

// Last-block finalisation: every block of a reducing kernel writes its partials, then counts
// itself done; the last block to finish (it sees every other block's partials after the fence)
// runs the scalar step that would otherwise be a separate one-block launch, and re-arms the
// counter for the next launch.  Call with the whole block; returns true in the last block.
__device__ __forceinline__ bool last_block(unsigned int *counter) {
    __shared__ unsigned int s_last;
    __threadfence();  // every thread's partial writes, before the block counts itself done
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    const bool last = s_last != 0;
    if (last) __threadfence();
    return last;
}

// Arguments of the CG scalar steps when a reducing kernel finalises them in its last block.
struct CgFin {
    double *S;
    int *state, *want, *iters;
    double *hist;
    CgCtl *ctl;
    int mode;
};

template <bool GEN>
__device__ void fin_gamma_dev(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ state,
                              int *__restrict__ want, int *__restrict__ iters, double *__restrict__ hist_beta,
                              CgCtl *__restrict__ ctl, int mode);
template <bool GEN>
__device__ void fin_delta_dev(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ state,
                              const int *__restrict__ want, int *__restrict__ iters, double *__restrict__ hist_alpha,
                              CgCtl *__restrict__ ctl, int mode);

struct BandOffs {
    int off[343];
};

// ------------------------------------------------------------------ reductions
// Block partial of per-thread values: FP32 warp tree for FP32 data, FP64 above (and for FP64).
template <typename T>
__device__ __forceinline__ double block_sum(T v, double *sh) {
    double dv;
    if (sizeof(T) == 4) {
        float f = (float)v;
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
// acc + b x for a band value b and a vector entry x; for double-float vectors the FP32 band value
// multiplies exactly (TwoProd) and the sum is a double-float addition.
template <typename TB, typename TX>
__device__ __forceinline__ TX band_fma(TB b, TX x, TX acc) { return fma((TX)b, x, acc); }
template <>
__device__ __forceinline__ dfl band_fma<float, dfl>(float b, dfl x, dfl acc) {
    df_acc_fx(acc, b, x);
    return acc;
}

// u[r][j] = sum_o band[o][j] * x[r][j + off(o)]  (entries whose neighbour is off-grid are zero,
// so the neighbour index is only clamped to stay in memory).  Band in TB, vectors in TX.
// Optional partial dots per rhs: q0 = u.x, q1 = x.g.  `gate` skips the launch's work when set.
template <typename TB, typename TX, int RB>
__global__ void __launch_bounds__(CG_T) k_band_spmv(const TB *__restrict__ band, int nband, const TX *__restrict__ x,
                                                     TX *__restrict__ u, int64_t m, int R, BandOffs offs,
                                                     double *__restrict__ part, int NQ, const TX *__restrict__ g,
                                                     const int *__restrict__ gate, int Rtot, int r0) {
    if (gate && *gate) return;
    __shared__ double sh[CG_T / 32];
    TX dq0[RB], dq1[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) dq0[k] = dq1[k] = TX(0);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        TX acc[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k) acc[k] = TX(0);
        for (int o = 0; o < nband; ++o) {
            const TB b = band[(int64_t)o * m + j];
            int64_t nb = j + offs.off[o];
            nb = nb < 0 ? 0 : (nb >= m ? m - 1 : nb);
#pragma unroll
            for (int k = 0; k < RB; ++k)
                if (k < R) acc[k] = band_fma<TB, TX>(b, x[(int64_t)k * m + nb], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < RB; ++k)
            if (k < R) {
                u[(int64_t)k * m + j] = acc[k];
                if (part) {
                    const TX xv = x[(int64_t)k * m + j];
                    dq0[k] = fma(acc[k], xv, dq0[k]);
                    if (g) dq1[k] = fma(xv, g[(int64_t)k * m + j], dq1[k]);
                }
            }
    }
    if (!part) return;
    for (int k = 0; k < R && k < RB; ++k) {
        const double s0 = block_sum<TX>(dq0[k], sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + 0] = s0;
        if (NQ > 1) {
            const double s1 = block_sum<TX>(dq1[k], sh);
            if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + 1] = s1;
        }
    }
}

// Vectorised form for an FP32 band and FP32 vectors (the MIXED iterations).  Each thread owns 4
// consecutive nodes i0..i0+3: every diagonal is one aligned float4 of the band, streamed past L1
// (each band value is used once per launch), and the 7 neighbours along the last axis of all 4
// nodes are one 12-wide window of x, three aligned float4 per grid row (dz, dy) and rhs.  The
// row loop is not unrolled: its 7 independent float4 band loads are in flight together.  Needs
// m and M_{d-1} to be multiples of 4 so that every row start stays 16-byte aligned.
struct RowOffs {
    int base[49];  // offset of row (dz, dy) = (row / 7 - 3, row % 7 - 3); diagonal o = row * 7 + dx + 3
};

// Only the first `nwork` blocks (as many as are resident at once) do work; the others write
// zero partials so that the partial-sum layout stays one entry per launched block.
template <int RB>
struct Spmv4Occ {
    static constexpr int blocks = RB <= 1 ? 4 : (RB <= 2 ? 3 : 2);
};

template <int NROW, int RB>
__global__ void __launch_bounds__(CG_T, Spmv4Occ<RB>::blocks) k_band_spmv4(const float *__restrict__ band, const float *__restrict__ x,
                                                      float *__restrict__ u, int64_t m, int R, RowOffs rows,
                                                      double *__restrict__ part, int NQ, const float *__restrict__ g,
                                                      const int *__restrict__ gate, int Rtot, int r0, int nwork) {
    if (gate && *gate) return;
    __shared__ double sh[CG_T / 32];
    if ((int)blockIdx.x >= nwork) {
        if (part && threadIdx.x == 0)
            for (int k = 0; k < R && k < RB; ++k)
                for (int q = 0; q < NQ && q < 2; ++q) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + q] = 0.0;
        return;
    }
    float dq0[RB], dq1[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) dq0[k] = dq1[k] = 0.f;
    const int64_t nquad = m >> 2;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nquad; t += (int64_t)nwork * blockDim.x) {
        const int64_t i0 = t << 2;
        float acc[RB][4];
#pragma unroll
        for (int k = 0; k < RB; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[k][q] = 0.f;
#pragma unroll 1
        for (int row = 0; row < NROW; ++row) {
            float4 b[7];
#pragma unroll
            for (int e = 0; e < 7; ++e) b[e] = __ldcs(reinterpret_cast<const float4 *>(band + (int64_t)(row * 7 + e) * m + i0));
            const int64_t w0 = i0 + rows.base[row] - 4;  // window x[w0 .. w0 + 11]
            const bool inside = w0 >= 0 && w0 + 12 <= m;
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                if (k < R) {
                    const float *xk = x + (int64_t)k * m;
                    float v[12];
                    if (inside) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float4 f = __ldg(reinterpret_cast<const float4 *>(xk + w0) + c);
                            v[4 * c] = f.x;
                            v[4 * c + 1] = f.y;
                            v[4 * c + 2] = f.z;
                            v[4 * c + 3] = f.w;
                        }
                    } else {
                        // grid ends: off-grid neighbours have zero band entries; read nothing there
#pragma unroll
                        for (int j = 0; j < 12; ++j) v[j] = (w0 + j >= 0 && w0 + j < m) ? __ldg(xk + w0 + j) : 0.f;
                    }
#pragma unroll
                    for (int e = 0; e < 7; ++e) {
                        acc[k][0] = fmaf(b[e].x, v[e + 1], acc[k][0]);
                        acc[k][1] = fmaf(b[e].y, v[e + 2], acc[k][1]);
                        acc[k][2] = fmaf(b[e].z, v[e + 3], acc[k][2]);
                        acc[k][3] = fmaf(b[e].w, v[e + 4], acc[k][3]);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < RB; ++k)
            if (k < R) {
                *reinterpret_cast<float4 *>(u + (int64_t)k * m + i0) = make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
                if (part) {
                    const float4 xv = __ldg(reinterpret_cast<const float4 *>(x + (int64_t)k * m + i0));
                    dq0[k] = fmaf(acc[k][0], xv.x, dq0[k]);
                    dq0[k] = fmaf(acc[k][1], xv.y, dq0[k]);
                    dq0[k] = fmaf(acc[k][2], xv.z, dq0[k]);
                    dq0[k] = fmaf(acc[k][3], xv.w, dq0[k]);
                    if (g) {
                        const float4 gv = __ldg(reinterpret_cast<const float4 *>(g + (int64_t)k * m + i0));
                        dq1[k] = fmaf(xv.x, gv.x, dq1[k]);
                        dq1[k] = fmaf(xv.y, gv.y, dq1[k]);
                        dq1[k] = fmaf(xv.z, gv.z, dq1[k]);
                        dq1[k] = fmaf(xv.w, gv.w, dq1[k]);
                    }
                }
            }
    }
    if (!part) return;
    for (int k = 0; k < R && k < RB; ++k) {
        const double s0 = block_sum<float>(dq0[k], sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + 0] = s0;
        if (NQ > 1) {
            const double s1 = block_sum<float>(dq1[k], sh);
            if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + 1] = s1;
        }
    }
}

// Symmetric form for one FP32 right-hand side: W^T W is symmetric, so only the diagonals with
// offset >= 0 are read -- a contiguous suffix of the stored band (centre row dx = 0..3, then
// the 7 diagonals of every later row) -- about half the bytes.  The lower part of row i is
// entry (i - off, i) of the stored upper diagonal:  u_i += H_off[i - off] x[i - off].  A thread
// reads, per upper row, its 7 direct quads at i0 and two quads around i0 - rowbase per
// diagonal for the mirrored term; the mirrored quads are the direct quads of the thread
// rowbase/4 positions back, read at about the same time, so they come from L2.
// FIN 1 / 2: the last block to finish takes the CG gamma step (fin_gamma_dev, plain / GEN) from
// all blocks' partials (R = 1 layout).
template <int NROW, int FIN>
__global__ void __launch_bounds__(CG_T, 2) k_band_spmv4h(const float *__restrict__ hb, const float *__restrict__ x,
                                                          float *__restrict__ u, int64_t m, RowOffs rows,
                                                          double *__restrict__ part, int NQ, const float *__restrict__ g,
                                                          const int *__restrict__ gate, int Rtot, int r0, int nwork,
                                                          CgFin fin) {
    if (gate && *gate) return;
    __shared__ double sh[CG_T / 32];
    if ((int)blockIdx.x >= nwork) {
        if (part && threadIdx.x == 0)
            for (int q = 0; q < NQ && q < 2; ++q) part[(int64_t)blockIdx.x * NQ * Rtot + r0 * NQ + q] = 0.0;
        if (FIN && last_block(&fin.ctl->fin_cnt[0])) {
            fin_gamma_dev<FIN == 2>(part, gridDim.x, fin.S, fin.state, fin.want, fin.iters, fin.hist, fin.ctl, fin.mode);
            if (threadIdx.x == 0) fin.ctl->fin_cnt[0] = 0;
        }
        return;
    }
    constexpr int C = NROW / 2;  // centre row
    float dq0 = 0.f, dq1 = 0.f;
    const int64_t nquad = m >> 2;
    // quad at j (multiple of 4), zero off the ends; read-only loads that ask L2 to fetch the
    // surrounding 256 B (a warp's band quads are contiguous, so DRAM sees larger bursts)
    auto ld4 = [&](const float *base, int64_t j) -> float4 {
        if (j >= 0 && j + 4 <= m) {
            float4 r;
            asm volatile("ld.global.nc.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                         : "l"(base + j));
            return r;
        }
        return make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto xwin = [&](int64_t w0, float v[12]) {  // x[w0 .. w0 + 11], zero off the ends
        if (w0 >= 0 && w0 + 12 <= m) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4 f = __ldg(reinterpret_cast<const float4 *>(x + w0) + c);
                v[4 * c] = f.x; v[4 * c + 1] = f.y; v[4 * c + 2] = f.z; v[4 * c + 3] = f.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 12; ++j) v[j] = (w0 + j >= 0 && w0 + j < m) ? __ldg(x + w0 + j) : 0.f;
        }
    };
    auto comp = [](const float4 &f, int q) { return q == 0 ? f.x : (q == 1 ? f.y : (q == 2 ? f.z : f.w)); };
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nquad; t += (int64_t)nwork * blockDim.x) {
        const int64_t i0 = t << 2;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        {
            // centre row: direct dx = 0..3, mirrored dx = 1..3
            float v[12];
            xwin(i0 - 4, v);
            float4 hc[4], hp[4];
#pragma unroll
            for (int dx = 0; dx < 4; ++dx) {
                hc[dx] = ld4(hb + (int64_t)dx * m, i0);
                hp[dx] = dx ? ld4(hb + (int64_t)dx * m, i0 - 4) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int dx = 0; dx < 4; ++dx)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[q] = fmaf(comp(hc[dx], q), v[q + dx + 4], acc[q]);
                    if (dx > 0) {
                        const int j = q - dx;  // mirrored entry at i0 + j
                        const float h = j < 0 ? comp(hp[dx], j + 4) : comp(hc[dx], j);
                        acc[q] = fmaf(h, v[j + 4], acc[q]);
                    }
                }
        }
#pragma unroll 2
        for (int u_ = 0; u_ < C; ++u_) {
            const int row = C + 1 + u_;
            const int64_t rb = rows.base[row];
            const float *hrow = hb + (int64_t)(4 + u_ * 7) * m;
            {
                float4 dq[7];
#pragma unroll
                for (int e = 0; e < 7; ++e) dq[e] = ld4(hrow + (int64_t)e * m, i0);
                float v[12];
                xwin(i0 + rb - 4, v);
#pragma unroll
                for (int e = 0; e < 7; ++e)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] = fmaf(comp(dq[e], q), v[q + e + 1], acc[q]);
            }
            float vm[12];
            xwin(i0 - rb - 4, vm);
            const int64_t j0 = i0 - rb;
#pragma unroll
            for (int e = 0; e < 7; ++e) {
                // entries j0 + 3 - e + q, q = 0..3, of diagonal e
                const float *hd = hrow + (int64_t)e * m;
                const float4 qa = e > 3 ? ld4(hd, j0 - 4) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 qb = ld4(hd, j0);
                const float4 qc = e < 3 ? ld4(hd, j0 + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int tt = 3 - e + q;  // offset from j0, in [-3, 6]
                    const float h = tt < 0 ? comp(qa, tt + 4) : (tt < 4 ? comp(qb, tt) : comp(qc, tt - 4));
                    acc[q] = fmaf(h, vm[tt + 4], acc[q]);
                }
            }
        }
        *reinterpret_cast<float4 *>(u + i0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        if (part) {
            const float4 xv = __ldg(reinterpret_cast<const float4 *>(x + i0));
            dq0 = fmaf(acc[0], xv.x, dq0);
            dq0 = fmaf(acc[1], xv.y, dq0);
            dq0 = fmaf(acc[2], xv.z, dq0);
            dq0 = fmaf(acc[3], xv.w, dq0);
            if (g) {
                const float4 gv = __ldg(reinterpret_cast<const float4 *>(g + i0));
                dq1 = fmaf(xv.x, gv.x, dq1);
                dq1 = fmaf(xv.y, gv.y, dq1);
                dq1 = fmaf(xv.z, gv.z, dq1);
                dq1 = fmaf(xv.w, gv.w, dq1);
            }
        }
    }
    if (!part) return;
    const double s0 = block_sum<float>(dq0, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + r0 * NQ + 0] = s0;
    if (NQ > 1) {
        const double s1 = block_sum<float>(dq1, sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + r0 * NQ + 1] = s1;
    }
    if (FIN && last_block(&fin.ctl->fin_cnt[0])) {
        fin_gamma_dev<FIN == 2>(part, gridDim.x, fin.S, fin.state, fin.want, fin.iters, fin.hist, fin.ctl, fin.mode);
        if (threadIdx.x == 0) fin.ctl->fin_cnt[0] = 0;
    }
}

static int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 1;
    }
    return n;
}

// The same vectorised form for FP64 vectors (true residuals, W^T x, FP64 solves) and FP64 bands:
// 4 nodes per thread, the band quad and the 12-wide x window loaded as 16-byte vectors.
template <typename T>
struct Quad {
    T v[4];
};

template <typename T>
__device__ __forceinline__ Quad<T> ld_quad(const T *p, bool stream);
template <>
__device__ __forceinline__ Quad<float> ld_quad<float>(const float *p, bool stream) {
    const float4 f = stream ? __ldcs(reinterpret_cast<const float4 *>(p)) : __ldg(reinterpret_cast<const float4 *>(p));
    return Quad<float>{{f.x, f.y, f.z, f.w}};
}
template <>
__device__ __forceinline__ Quad<double> ld_quad<double>(const double *p, bool stream) {
    const double2 a = stream ? __ldcs(reinterpret_cast<const double2 *>(p)) : __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = stream ? __ldcs(reinterpret_cast<const double2 *>(p) + 1) : __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return Quad<double>{{a.x, a.y, b.x, b.y}};
}

template <>
__device__ __forceinline__ Quad<dfl> ld_quad<dfl>(const dfl *p, bool stream) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    const float4 a = stream ? __ldcs(q) : __ldg(q);
    const float4 b = stream ? __ldcs(q + 1) : __ldg(q + 1);
    return Quad<dfl>{{dfl(a.x, a.y), dfl(a.z, a.w), dfl(b.x, b.y), dfl(b.z, b.w)}};
}

template <typename T>
__device__ __forceinline__ void st_quad(T *p, const T v[4]);
template <>
__device__ __forceinline__ void st_quad<dfl>(dfl *p, const dfl v[4]) {
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    reinterpret_cast<float4 *>(p)[1] = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
}
template <>
__device__ __forceinline__ void st_quad<float>(float *p, const float v[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st_quad<double>(double *p, const double v[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// Band-product accumulator: FMA in TX, or the lazily normalised double-float sum for an FP32
// band on double-float vectors.
template <typename TB, typename TX>
struct BandAcc {
    TX v;
    __device__ __forceinline__ void zero() { v = TX(0); }
    __device__ __forceinline__ void add(TB b, TX x) { v = fma((TX)b, x, v); }
    __device__ __forceinline__ TX value() const { return v; }
};
template <>
struct BandAcc<float, dfl> {
    dacc a;
    __device__ __forceinline__ void zero() { dacc_zero(a); }
    __device__ __forceinline__ void add(float b, dfl x) { dacc_add_fx(a, b, x); }
    __device__ __forceinline__ dfl value() const { return dacc_value(a); }
};

template <typename TB, typename TX, int NROW, int RB>
__global__ void __launch_bounds__(CG_T, RB <= 2 ? 2 : 1) k_band_spmv4g(const TB *__restrict__ band, const TX *__restrict__ x,
                                                          TX *__restrict__ u, int64_t m, int R, RowOffs rows,
                                                          double *__restrict__ part, int NQ, const TX *__restrict__ g,
                                                          const int *__restrict__ gate, int Rtot, int r0, int nwork) {
    if (gate && *gate) return;
    __shared__ double sh[CG_T / 32];
    if ((int)blockIdx.x >= nwork) {
        if (part && threadIdx.x == 0)
            for (int k = 0; k < R && k < RB; ++k)
                for (int q = 0; q < NQ && q < 2; ++q) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + q] = 0.0;
        return;
    }
    TX dq0[RB], dq1[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) dq0[k] = dq1[k] = TX(0);
    const int64_t nquad = m >> 2;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nquad; t += (int64_t)nwork * blockDim.x) {
        const int64_t i0 = t << 2;
        BandAcc<TB, TX> acc[RB][4];
#pragma unroll
        for (int k = 0; k < RB; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[k][q].zero();
#pragma unroll 1
        for (int row = 0; row < NROW; ++row) {
            Quad<TB> b[7];
#pragma unroll
            for (int e = 0; e < 7; ++e) b[e] = ld_quad<TB>(band + (int64_t)(row * 7 + e) * m + i0, true);
            const int64_t w0 = i0 + rows.base[row] - 4;
            const bool inside = w0 >= 0 && w0 + 12 <= m;
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                if (k < R) {
                    const TX *xk = x + (int64_t)k * m;
                    TX v[12];
                    if (inside) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const Quad<TX> f = ld_quad<TX>(xk + w0 + 4 * c, false);
#pragma unroll
                            for (int q = 0; q < 4; ++q) v[4 * c + q] = f.v[q];
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 12; ++j) v[j] = (w0 + j >= 0 && w0 + j < m) ? xk[w0 + j] : TX(0);
                    }
#pragma unroll
                    for (int e = 0; e < 7; ++e)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[k][q].add(b[e].v[q], v[e + 1 + q]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < RB; ++k)
            if (k < R) {
                TX uv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) uv[q] = acc[k][q].value();
                st_quad<TX>(u + (int64_t)k * m + i0, uv);
                if (part) {
                    const Quad<TX> xv = ld_quad<TX>(x + (int64_t)k * m + i0, false);
#pragma unroll
                    for (int q = 0; q < 4; ++q) dq0[k] = fma(uv[q], xv.v[q], dq0[k]);
                    if (g) {
                        const Quad<TX> gv = ld_quad<TX>(g + (int64_t)k * m + i0, false);
#pragma unroll
                        for (int q = 0; q < 4; ++q) dq1[k] = fma(xv.v[q], gv.v[q], dq1[k]);
                    }
                }
            }
    }
    if (!part) return;
    for (int k = 0; k < R && k < RB; ++k) {
        const double s0 = block_sum<TX>(dq0[k], sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + 0] = s0;
        if (NQ > 1) {
            const double s1 = block_sum<TX>(dq1[k], sh);
            if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ * Rtot + (r0 + k) * NQ + 1] = s1;
        }
    }
}

// The half-band product for one double-float right-hand side (the MIXED iterations): the same
// traversal as k_band_spmv4h (direct quads of the stored upper diagonals at i0, mirrored quads
// around i0 - rowbase), with x and u as double-float values (a 12-wide window is six 16-byte
// loads) and every band product accumulated in a lazily normalised double-float sum (dacc).
// The band stays FP32, so the bytes read per launch are the FP32 half band plus 16 B per node
// for x and u.
template <int NROW, int FIN>
__global__ void __launch_bounds__(CG_T, 2) k_band_spmv4hd(const float *__restrict__ hb, const dfl *__restrict__ x,
                                                           dfl *__restrict__ u, int64_t m, RowOffs rows,
                                                           double *__restrict__ part, int NQ, const dfl *__restrict__ g,
                                                           const int *__restrict__ gate, int nwork, CgFin fin) {
    if (gate && *gate) return;
    __shared__ double sh[CG_T / 32];
    if ((int)blockIdx.x >= nwork) {
        if (part && threadIdx.x == 0)
            for (int q = 0; q < NQ && q < 2; ++q) part[(int64_t)blockIdx.x * NQ + q] = 0.0;
        if (FIN && last_block(&fin.ctl->fin_cnt[0])) {
            fin_gamma_dev<FIN == 2>(part, gridDim.x, fin.S, fin.state, fin.want, fin.iters, fin.hist, fin.ctl, fin.mode);
            if (threadIdx.x == 0) fin.ctl->fin_cnt[0] = 0;
        }
        return;
    }
    constexpr int C = NROW / 2;  // centre row
    dfl dq0 = dfl(0), dq1 = dfl(0);
    const int64_t nquad = m >> 2;
    auto ld4 = [&](const float *base, int64_t j) -> float4 {
        if (j >= 0 && j + 4 <= m) {
            float4 r;
            asm volatile("ld.global.nc.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                         : "l"(base + j));
            return r;
        }
        return make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto xwin = [&](int64_t w0, dfl v[12]) {  // x[w0 .. w0 + 11], zero off the ends
        if (w0 >= 0 && w0 + 12 <= m) {
            const float4 *q = reinterpret_cast<const float4 *>(x + w0);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const float4 f = __ldg(q + c);
                v[2 * c] = dfl(f.x, f.y);
                v[2 * c + 1] = dfl(f.z, f.w);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 12; ++j) v[j] = (w0 + j >= 0 && w0 + j < m) ? x[w0 + j] : dfl(0);
        }
    };
    auto comp = [](const float4 &f, int q) { return q == 0 ? f.x : (q == 1 ? f.y : (q == 2 ? f.z : f.w)); };
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nquad; t += (int64_t)nwork * blockDim.x) {
        const int64_t i0 = t << 2;
        dacc acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) dacc_zero(acc[q]);
        {
            dfl v[12];
            xwin(i0 - 4, v);
            float4 hc[4], hp[4];
#pragma unroll
            for (int dx = 0; dx < 4; ++dx) {
                hc[dx] = ld4(hb + (int64_t)dx * m, i0);
                hp[dx] = dx ? ld4(hb + (int64_t)dx * m, i0 - 4) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int dx = 0; dx < 4; ++dx)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    dacc_add_fx(acc[q], comp(hc[dx], q), v[q + dx + 4]);
                    if (dx > 0) {
                        const int j = q - dx;
                        const float h = j < 0 ? comp(hp[dx], j + 4) : comp(hc[dx], j);
                        dacc_add_fx(acc[q], h, v[j + 4]);
                    }
                }
        }
#pragma unroll 1
        for (int u_ = 0; u_ < C; ++u_) {
            const int row = C + 1 + u_;
            const int64_t rb = rows.base[row];
            const float *hrow = hb + (int64_t)(4 + u_ * 7) * m;
            {
                float4 dq[7];
#pragma unroll
                for (int e = 0; e < 7; ++e) dq[e] = ld4(hrow + (int64_t)e * m, i0);
                dfl v[12];
                xwin(i0 + rb - 4, v);
#pragma unroll
                for (int e = 0; e < 7; ++e)
#pragma unroll
                    for (int q = 0; q < 4; ++q) dacc_add_fx(acc[q], comp(dq[e], q), v[q + e + 1]);
            }
            dfl vm[12];
            xwin(i0 - rb - 4, vm);
            const int64_t j0 = i0 - rb;
#pragma unroll
            for (int e = 0; e < 7; ++e) {
                const float *hd = hrow + (int64_t)e * m;
                const float4 qa = e > 3 ? ld4(hd, j0 - 4) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 qb = ld4(hd, j0);
                const float4 qc = e < 3 ? ld4(hd, j0 + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int tt = 3 - e + q;
                    const float h = tt < 0 ? comp(qa, tt + 4) : (tt < 4 ? comp(qb, tt) : comp(qc, tt - 4));
                    dacc_add_fx(acc[q], h, vm[tt + 4]);
                }
            }
        }
        dfl ur[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) ur[q] = dacc_value(acc[q]);
        float4 *uq = reinterpret_cast<float4 *>(u + i0);
        uq[0] = make_float4(ur[0].hi, ur[0].lo, ur[1].hi, ur[1].lo);
        uq[1] = make_float4(ur[2].hi, ur[2].lo, ur[3].hi, ur[3].lo);
        if (part) {
            const Quad<dfl> xv = ld_quad<dfl>(x + i0, false);
#pragma unroll
            for (int q = 0; q < 4; ++q) dq0 = fma(ur[q], xv.v[q], dq0);
            if (g) {
                const Quad<dfl> gv = ld_quad<dfl>(g + i0, false);
#pragma unroll
                for (int q = 0; q < 4; ++q) dq1 = fma(xv.v[q], gv.v[q], dq1);
            }
        }
    }
    if (!part) return;
    const double s0 = block_sum<dfl>(dq0, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ + 0] = s0;
    if (NQ > 1) {
        const double s1 = block_sum<dfl>(dq1, sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NQ + 1] = s1;
    }
    if (FIN && last_block(&fin.ctl->fin_cnt[0])) {
        fin_gamma_dev<FIN == 2>(part, gridDim.x, fin.S, fin.state, fin.want, fin.iters, fin.hist, fin.ctl, fin.mode);
        if (threadIdx.x == 0) fin.ctl->fin_cnt[0] = 0;
    }
}

static bool spmv4_ok(const fkski_grid &g, int64_t m, const void *band, const void *x, const void *u, const void *gv) {
    if ((m & 3) != 0 || (g.M[g.d - 1] & 3) != 0) return false;
    const uintptr_t a = (uintptr_t)band | (uintptr_t)x | (uintptr_t)u | (uintptr_t)gv;
    return (a & 15) == 0;
}

static RowOffs make_rows(const fkski_grid &g) {
    RowOffs ro;
    memset(&ro, 0, sizeof(ro));
    if (g.d == 3) {
        for (int row = 0; row < 49; ++row)
            ro.base[row] = (int)((row / 7 - 3) * g.M[1] * g.M[2] + (row % 7 - 3) * g.M[2]);
    } else if (g.d == 2) {
        for (int row = 0; row < 7; ++row) ro.base[row] = (int)((row - 3) * g.M[1]);
    }
    return ro;
}

template <int NROW>
static void launch_spmv4_rows(const float *band, const float *x, float *u, int64_t m, int R, const RowOffs &ro,
                              double *part, int NQ, const float *gv, const int *gate, int nblocks, int Rtot, int r0,
                              cudaStream_t s) {
#define FK_SPMV4(RBV) \
    k_band_spmv4<NROW, RBV><<<nblocks, CG_T, 0, s>>>(band, x, u, m, R, ro, part, NQ, gv, gate, Rtot, r0, \
                                                      std::min(nblocks, num_sms() * Spmv4Occ<RBV>::blocks))
    if (R <= 1) FK_SPMV4(1);
    else if (R <= 2) FK_SPMV4(2);
    else if (R <= 4) FK_SPMV4(4);
    else FK_SPMV4(8);
#undef FK_SPMV4
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

template <typename TB, typename TX>
static int launch_spmv(const TB *band, const fkski_grid &g, const TX *x, TX *u, int64_t m, int R, double *part, int NQ,
                       const TX *gv, const int *gate, int nblocks, cudaStream_t s) {
    if constexpr (std::is_same<TB, float>::value && std::is_same<TX, float>::value) {
        if (spmv4_ok(g, m, band, x, u, gv)) {
            const RowOffs ro = make_rows(g);
            if (R == 1) {
                // one rhs: symmetric half (the stored band from the centre row's dx = 0 onwards)
                const int nrow = g.d == 3 ? 49 : (g.d == 2 ? 7 : 1);
                const float *hb = band + (int64_t)((nrow / 2) * 7 + 3) * m;
                const int nwork = std::min(nblocks, num_sms() * 2);
                if (g.d == 3) k_band_spmv4h<49, 0><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, 1, 0, nwork, CgFin{});
                else if (g.d == 2) k_band_spmv4h<7, 0><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, 1, 0, nwork, CgFin{});
                else k_band_spmv4h<1, 0><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, 1, 0, nwork, CgFin{});
                FK_LAUNCH();
                return FKSKI_OK;
            }
            // rhs in even groups of at most 8: the band is read once per group
            const int ng = (int)cdiv(R, 8), per = (int)cdiv(R, ng);
            for (int r0 = 0; r0 < R; r0 += per) {
                const int Rb = std::min(per, R - r0);
                const float *xb = x + (int64_t)r0 * m;
                float *ub = u + (int64_t)r0 * m;
                const float *gb = gv ? gv + (int64_t)r0 * m : nullptr;
                if (g.d == 3) launch_spmv4_rows<49>(band, xb, ub, m, Rb, ro, part, NQ, gb, gate, nblocks, R, r0, s);
                else if (g.d == 2) launch_spmv4_rows<7>(band, xb, ub, m, Rb, ro, part, NQ, gb, gate, nblocks, R, r0, s);
                else launch_spmv4_rows<1>(band, xb, ub, m, Rb, ro, part, NQ, gb, gate, nblocks, R, r0, s);
                FK_LAUNCH();
            }
            return FKSKI_OK;
        }
    }
    if constexpr (std::is_same<TB, float>::value && std::is_same<TX, dfl>::value) {
        if (R == 1 && spmv4_ok(g, m, band, x, u, gv)) {
            // one double-float rhs: the symmetric half band, as for FP32
            const RowOffs ro = make_rows(g);
            const int nrow = g.d == 3 ? 49 : (g.d == 2 ? 7 : 1);
            const float *hb = band + (int64_t)((nrow / 2) * 7 + 3) * m;
            const int nwork = std::min(nblocks, num_sms() * 2);
            if (g.d == 3) k_band_spmv4hd<49, 0><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, nwork, CgFin{});
            else if (g.d == 2) k_band_spmv4hd<7, 0><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, nwork, CgFin{});
            else k_band_spmv4hd<1, 0><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, nwork, CgFin{});
            FK_LAUNCH();
            return FKSKI_OK;
        }
    }
    if constexpr (!(std::is_same<TB, float>::value && std::is_same<TX, float>::value)) {
        if (spmv4_ok(g, m, band, x, u, gv)) {
            const RowOffs ro = make_rows(g);
            // rhs in even groups of at most 4 (FP64 accumulators); double-float rhs in groups of
            // at most 2 (128 registers, two CTAs per SM; four rhs need 168 registers and one CTA
            // per SM: 1.82 against 1.71 ms per 17-rhs gradient iteration on a 64^3 grid)
            const int cap = std::is_same<TX, dfl>::value ? 2 : 4;
            const int ng = (int)cdiv(R, cap), per = (int)cdiv(R, ng);
            for (int r0 = 0; r0 < R; r0 += per) {
                const int Rb = std::min(per, R - r0);
                const int nwork = std::min(nblocks, num_sms() * (Rb <= 2 ? 2 : 1));
                const TX *xb = x + (int64_t)r0 * m;
                TX *ub = u + (int64_t)r0 * m;
                const TX *gb2 = gv ? gv + (int64_t)r0 * m : nullptr;
#define FK_SPMV4G(NR, RBV) \
    k_band_spmv4g<TB, TX, NR, RBV><<<nblocks, CG_T, 0, s>>>(band, xb, ub, m, Rb, ro, part, NQ, gb2, gate, R, r0, nwork)
#define FK_SPMV4G_R(NR)                   \
    do {                                  \
        if (Rb <= 1) FK_SPMV4G(NR, 1);    \
        else if (Rb <= 2) FK_SPMV4G(NR, 2); \
        else FK_SPMV4G(NR, 4);            \
    } while (0)
                if (g.d == 3) FK_SPMV4G_R(49);
                else if (g.d == 2) FK_SPMV4G_R(7);
                else FK_SPMV4G_R(1);
#undef FK_SPMV4G_R
#undef FK_SPMV4G
                FK_LAUNCH();
            }
            return FKSKI_OK;
        }
    }
    const BandOffs bo = make_offs(g);
    const int nb = (int)ipow(7, g.d);
    for (int r0 = 0; r0 < R; r0 += 32) {
        const int Rb = std::min(32, R - r0);
        const TX *xb = x + (int64_t)r0 * m;
        TX *ub = u + (int64_t)r0 * m;
        const TX *gb = gv ? gv + (int64_t)r0 * m : nullptr;
#define FK_SPMV(RBV) \
    k_band_spmv<TB, TX, RBV><<<nblocks, CG_T, 0, s>>>(band, nb, xb, ub, m, Rb, bo, part, NQ, gb, gate, R, r0)
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

// One FP32 rhs: the half-band product with the CG gamma step taken by its last block (returns
// FKSKI_E_UNSUPPORTED, launching nothing, where the half-band kernel does not apply).
template <bool GEN>
static int launch_spmvh_fin(const float *band, const fkski_grid &g, const float *x, float *u, int64_t m,
                            double *part, int NQ, const float *gv, const int *gate, int nblocks, const CgFin &fin,
                            cudaStream_t s) {
    if (!spmv4_ok(g, m, band, x, u, gv)) return FKSKI_E_UNSUPPORTED;
    const RowOffs ro = make_rows(g);
    const int nrow = g.d == 3 ? 49 : (g.d == 2 ? 7 : 1);
    const float *hb = band + (int64_t)((nrow / 2) * 7 + 3) * m;
    const int nwork = std::min(nblocks, num_sms() * 2);
    constexpr int F = GEN ? 2 : 1;
    if (g.d == 3) k_band_spmv4h<49, F><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, 1, 0, nwork, fin);
    else if (g.d == 2) k_band_spmv4h<7, F><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, 1, 0, nwork, fin);
    else k_band_spmv4h<1, F><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, 1, 0, nwork, fin);

    FK_LAUNCH();
    return FKSKI_OK;
}

// The same for one double-float rhs (FP32 band).
template <bool GEN>
static int launch_spmvh_fin(const float *band, const fkski_grid &g, const dfl *x, dfl *u, int64_t m, double *part,
                            int NQ, const dfl *gv, const int *gate, int nblocks, const CgFin &fin, cudaStream_t s) {
    if (!spmv4_ok(g, m, band, x, u, gv)) return FKSKI_E_UNSUPPORTED;
    const RowOffs ro = make_rows(g);
    const int nrow = g.d == 3 ? 49 : (g.d == 2 ? 7 : 1);
    const float *hb = band + (int64_t)((nrow / 2) * 7 + 3) * m;
    const int nwork = std::min(nblocks, num_sms() * 2);
    constexpr int F = GEN ? 2 : 1;
    if (g.d == 3) k_band_spmv4hd<49, F><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, nwork, fin);
    else if (g.d == 2) k_band_spmv4hd<7, F><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, nwork, fin);
    else k_band_spmv4hd<1, F><<<nblocks, CG_T, 0, s>>>(hb, x, u, m, ro, part, NQ, gv, gate, nwork, fin);
    FK_LAUNCH();
    return FKSKI_OK;
}

// ------------------------------------------------------------------ small vector kernels
template <typename TI, typename TO>
__global__ void k_convert_t(const TI *__restrict__ in, TO *__restrict__ out, int64_t n, double c) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (TO)(c * (double)in[e]);
}

template <typename T>
__global__ void k_convert(const void *__restrict__ in, int in_dbl, T *__restrict__ out, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = in_dbl ? (T)((const double *)in)[e] : (T)((const float *)in)[e];
}

// out[r][i] = x[r][i] + c_r g[r][i]; c_r = S[F * R + r] or the constant c0.  FP64 result.
template <typename TG>
__global__ void k_axpy64(const double *__restrict__ x, const TG *__restrict__ g, double *__restrict__ out, int64_t m,
                         int R, const double *__restrict__ S, int F, double c0) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / m);
        const double c = S ? S[F * R + r] : c0;
        out[e] = fma(c, (double)g[e], x[e]);
    }
}

// partial dots of up to 4 pairs per rhs: part[blk][r][q] (NQ = 4 layout); unused pairs are null
template <typename TA, typename TB>
__global__ void __launch_bounds__(CG_T) k_dots4(const TA *__restrict__ a0, const TB *__restrict__ b0, const TA *__restrict__ a1,
                                                const TB *__restrict__ b1, const TA *__restrict__ a2, const TB *__restrict__ b2,
                                                const TA *__restrict__ a3, const TB *__restrict__ b3, int64_t m, int R,
                                                double *__restrict__ part, const int *__restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[CG_T / 32];
    using Acc = typename std::conditional<sizeof(TA) == 8 || sizeof(TB) == 8, double, float>::type;
    for (int r = 0; r < R; ++r) {
        Acc acc[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
            const int64_t e = (int64_t)r * m + j;
            acc[0] = fma((Acc)a0[e], (Acc)b0[e], acc[0]);
            if (a1) acc[1] = fma((Acc)a1[e], (Acc)b1[e], acc[1]);
            if (a2) acc[2] = fma((Acc)a2[e], (Acc)b2[e], acc[2]);
            if (a3) acc[3] = fma((Acc)a3[e], (Acc)b3[e], acc[3]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double s = block_sum<Acc>(acc[q], sh);
            if (threadIdx.x == 0) part[(int64_t)blockIdx.x * 4 * R + r * 4 + q] = s;
        }
    }
}

__global__ void k_pick(const double *__restrict__ in, int stride, int n, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[(int64_t)i * stride];
}

// out[r * NQ + q] = fixed-order sum of partials (one warp per (r, q))
__global__ void k_fin_sums(const double *__restrict__ part, int nparts, int R, int NQ, double *__restrict__ out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= R * NQ) return;
    const double s = warp_sum_partials(part, nparts, R, NQ, w / NQ, w % NQ);
    if ((threadIdx.x & 31) == 0) out[w] = s;
}

// ------------------------------------------------------------------ factorized CG kernels
// GEN = false: Alg. 5 (r = W r_hat).  GEN = true: Alg. 3's compressed form r = W r_hat + c^r b'
// with per-rhs base vector b', g = W^T b', kg = K_G g, rho' = ||b'||^2 (fields F_RHOP, F_GKG).
// The paper's Alg. 3 takes b' = r0 = b, r_hat_0 = 0.  Here b is first split as b = W b_hat + b'
// with b_hat a few CG steps on (W^T W) b_hat = W^T b, so b' is nearly orthogonal to range(W):
// its part outside range(W) is an exact eigenvector of A (eigenvalue sigma^2) and no longer
// cancels against in-span terms in the Claim 4 inner products (r_hat_0 = b_hat, c^r_0 = 1).
// A rhs with b' = 0 (g = 0, rho' = 0) runs Alg. 5's recurrence inside the same kernels.

// x_hat (FP64) += alpha p_hat;  r_hat -= alpha (z_hat + c^p kg)
template <typename T, bool GEN>
__global__ void __launch_bounds__(CG_T) k_cg_xr(int64_t m, int R, double *__restrict__ x, T *__restrict__ r,
                                                 const T *__restrict__ p, const T *__restrict__ z, const T *__restrict__ kg,
                                                 const double *__restrict__ S, const int *__restrict__ state,
                                                 const CgCtl *__restrict__ ctl) {
    if (ctl->all_done) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(e / m);
        if (state[rr] != RS_ACTIVE) continue;
        const double a = S[F_ALPHA * R + rr];
        x[e] = fma(a, (double)p[e], x[e]);
        const T at = (T)a;
        T zz = z[e];
        if (GEN) zz = fma((T)S[F_CP * R + rr], kg[e], zz);
        r[e] = fma(-at, zz, r[e]);
    }
}

// p = r + beta p; s = u + beta s; z = v + beta z; partial dots s.z, s.kg, p.g, z.g (layout NQ = 4);
// the last block then takes the alpha step (fin_delta_dev) from all blocks' partials.
template <typename T, bool GEN>
__global__ void __launch_bounds__(CG_T) k_cg_psz(int64_t m, int R, const T *__restrict__ r, const T *__restrict__ u,
                                                  const T *__restrict__ v, T *__restrict__ p, T *__restrict__ s, T *__restrict__ z,
                                                  const T *__restrict__ g, const T *__restrict__ kg,
                                                  double *__restrict__ part, CgFin fin) {
    const CgCtl *ctl = fin.ctl;
    const double *S = fin.S;
    const int *state = fin.state;
    if (ctl->all_done) return;
    __shared__ double sh[CG_T / 32];
    for (int rr = 0; rr < R; ++rr) {
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        if (state[rr] == RS_ACTIVE) {
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
                if (GEN) {
                    a1 = fma(sn, kg[e], a1);
                    a2 = fma(pn, g[e], a2);
                    a3 = fma(zn, g[e], a3);
                }
            }
        }
        const double t0 = block_sum<T>(a0, sh);
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        if (GEN) {
            t1 = block_sum<T>(a1, sh);
            t2 = block_sum<T>(a2, sh);
            t3 = block_sum<T>(a3, sh);
        }
        if (threadIdx.x == 0) {
            double *pp = part + (int64_t)blockIdx.x * 4 * R + rr * 4;
            pp[0] = t0; pp[1] = t1; pp[2] = t2; pp[3] = t3;
        }
    }
    if (last_block(&fin.ctl->fin_cnt[1])) {
        fin_delta_dev<GEN>(part, gridDim.x, fin.S, fin.state, fin.want, fin.iters, fin.hist, fin.ctl, fin.mode);
        if (threadIdx.x == 0) fin.ctl->fin_cnt[1] = 0;
    }
}

// gamma = <r, r> from u.r (q0) and r.g (q1) (Claim 4), after this iteration's x/r step
// (GEN: c^x, c^r follow the step first).  mode 0: iterate; 1: init (no step taken).
// Converged rhs become final (DOUBLE) or tentative, awaiting the true residual (MIXED).
template <bool GEN>
__device__ void fin_gamma_dev(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ state,
                              int *__restrict__ want, int *__restrict__ iters, double *__restrict__ hist_beta,
                              CgCtl *__restrict__ ctl, int mode) {
    if (ctl->all_done) return;
    const int R = ctl->R;
    const double s2 = ctl->sig2;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NQ = GEN ? 2 : 1;
    for (int r = w; r < R; r += blockDim.x >> 5) {
        const double ur = warp_sum_partials(part, nparts, R, NQ, r, 0);
        const double rg = GEN ? warp_sum_partials(part, nparts, R, NQ, r, 1) : 0.0;
        if (lane != 0 || state[r] != RS_ACTIVE) continue;
        double cr = 0.0;
        if (GEN) {
            if (mode == 0) {
                const double a = S[F_ALPHA * R + r], cp0 = S[F_CP * R + r];
                S[F_CX * R + r] += a * cp0;
                cr = S[F_CR * R + r] - a * s2 * cp0;
            } else {
                cr = S[F_CR * R + r];
            }
            S[F_CR * R + r] = cr;
        }
        const double g = ur + (GEN ? 2.0 * cr * rg + cr * cr * S[F_RHOP * R + r] : 0.0);
        S[F_RES * R + r] = g;
        S[F_GNEW * R + r] = g;
        if (mode == 1) S[F_GLAST * R + r] = g;
        if (!isfinite(g)) {
            state[r] = RS_FINAL;
            iters[r] = ctl->iter;
            atomicOr(&ctl->status, ST_BREAKDOWN);
            continue;
        }
        if (g <= S[F_EPS * R + r]) {
            state[r] = ctl->replace ? RS_TENTATIVE : RS_FINAL;
            iters[r] = mode == 1 ? 0 : ctl->iter + 1;
            continue;
        }
        if (ctl->replace && g < ctl->delta2 * S[F_GLAST * R + r]) want[r] = 1;
        if (mode == 1) {
            S[F_BETA * R + r] = 0.0;
        } else {
            const double be = g / S[F_GAMMA * R + r];
            S[F_BETA * R + r] = be;
            hist_beta[(int64_t)ctl->iter * R + r] = be;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1, conf = 1;
        for (int r = 0; r < R; ++r) {
            all &= state[r] != RS_ACTIVE;
            conf &= state[r] == RS_FINAL;
        }
        ctl->all_done = all;
        ctl->all_conf = conf;
    }
}

template <bool GEN>
__global__ void k_cg_fin_gamma(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ state,
                               int *__restrict__ want, int *__restrict__ iters, double *__restrict__ hist_beta,
                               CgCtl *__restrict__ ctl, int mode) {
    fin_gamma_dev<GEN>(part, nparts, S, state, want, iters, hist_beta, ctl, mode);
}

// alpha = gamma / <p, A p> (Claim 4 terms for GEN) for the next step.  mode 0: after an
// iteration (records the next alpha, advances the counter); 1: init.
template <bool GEN>
__device__ void fin_delta_dev(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ state,
                              const int *__restrict__ want, int *__restrict__ iters, double *__restrict__ hist_alpha,
                              CgCtl *__restrict__ ctl, int mode) {
    if (ctl->all_done) return;
    const int R = ctl->R;
    const double s2 = ctl->sig2;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = mode == 0 ? ctl->iter + 1 : ctl->iter;
    for (int r = w; r < R; r += blockDim.x >> 5) {
        const double sz = warp_sum_partials(part, nparts, R, 4, r, 0);
        const double skg = GEN ? warp_sum_partials(part, nparts, R, 4, r, 1) : 0.0;
        const double pg = GEN ? warp_sum_partials(part, nparts, R, 4, r, 2) : 0.0;
        const double zg = GEN ? warp_sum_partials(part, nparts, R, 4, r, 3) : 0.0;
        if (lane != 0 || state[r] != RS_ACTIVE) continue;
        double den = sz;
        if (GEN) {
            const double cp = S[F_CR * R + r] + S[F_BETA * R + r] * S[F_CP * R + r];
            const double cq = s2 * cp;
            den += cp * skg + cq * pg + cp * zg + cp * cp * S[F_GKG * R + r] + cp * cq * S[F_RHOP * R + r];
            S[F_CP * R + r] = cp;
        }
        S[F_DELTA * R + r] = den;
        if (!(den > 0.0) || !isfinite(den)) {
            state[r] = RS_FINAL;
            iters[r] = k;
            atomicOr(&ctl->status, ST_BREAKDOWN);
            continue;
        }
        const double gn = S[F_GNEW * R + r];
        const double a = gn / den;
        S[F_ALPHA * R + r] = a;
        S[F_GAMMA * R + r] = gn;
        if (k < ctl->maxiter) hist_alpha[(int64_t)k * R + r] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (mode == 0) ctl->iter += 1;
        int all = 1, conf = 1, rep = 0;
        for (int r = 0; r < R; ++r) {
            all &= state[r] != RS_ACTIVE;
            conf &= state[r] == RS_FINAL;
            rep |= want[r] || state[r] == RS_TENTATIVE;
        }
        if (ctl->iter >= ctl->maxiter) {
            all = 1;  // stop iterating
            if (ctl->replace) {
                rep = 1;  // the replacement pass confirms or finalises
            } else {
                for (int r = 0; r < R; ++r)
                    if (state[r] != RS_FINAL) { state[r] = RS_FINAL; iters[r] = ctl->maxiter; }
                conf = 1;
            }
        }
        ctl->all_done = all;
        ctl->all_conf = conf;
        ctl->any_rep = rep;
    }
}


// After a residual replacement (MIXED): gamma from the true residual for the flagged rhs;
// finish those that meet the tolerance, resume the others with alpha = gamma / <p, A p>
// (p, s, z unchanged).  Finalises everything at maxiter.
template <bool GEN>
__global__ void k_cg_fin_replace(const double *__restrict__ part, int nparts, double *__restrict__ S, int *__restrict__ state,
                                 int *__restrict__ want, int *__restrict__ iters, double *__restrict__ hist_alpha,
                                 CgCtl *__restrict__ ctl) {
    if (ctl->all_conf) return;
    const int R = ctl->R;
    const double s2 = ctl->sig2;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NQ = GEN ? 2 : 1;
    for (int r = w; r < R; r += blockDim.x >> 5) {
        const double ur = warp_sum_partials(part, nparts, R, NQ, r, 0);
        const double rg = GEN ? warp_sum_partials(part, nparts, R, NQ, r, 1) : 0.0;
        if (lane != 0) continue;
        const int stt = state[r];
        if (stt == RS_FINAL || !(want[r] || stt == RS_TENTATIVE)) continue;
        want[r] = 0;
        double cr = 0.0;
        if (GEN) {
            cr = 1.0 - s2 * S[F_CX * R + r];
            S[F_CR * R + r] = cr;
        }
        const double g = ur + (GEN ? 2.0 * cr * rg + cr * cr * S[F_RHOP * R + r] : 0.0);
        S[F_RES * R + r] = g;
        S[F_GLAST * R + r] = g;
        S[F_GAMMA * R + r] = g;
        S[F_GNEW * R + r] = g;
        if (!isfinite(g)) {
            state[r] = RS_FINAL;
            atomicOr(&ctl->status, ST_BREAKDOWN);
            continue;
        }
        if (g <= S[F_EPS * R + r]) {
            if (stt == RS_ACTIVE) iters[r] = ctl->iter;
            state[r] = RS_FINAL;
            continue;
        }
        state[r] = RS_ACTIVE;
        const double den = S[F_DELTA * R + r];
        if (!(den > 0.0)) {
            state[r] = RS_FINAL;
            atomicOr(&ctl->status, ST_BREAKDOWN);
            continue;
        }
        const double a = g / den;
        S[F_ALPHA * R + r] = a;
        if (ctl->iter < ctl->maxiter) hist_alpha[(int64_t)ctl->iter * R + r] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1, conf = 1;
        if (ctl->iter >= ctl->maxiter)
            for (int r = 0; r < R; ++r)
                if (state[r] != RS_FINAL) { state[r] = RS_FINAL; iters[r] = ctl->maxiter; }
        for (int r = 0; r < R; ++r) {
            all &= state[r] != RS_ACTIVE;
            conf &= state[r] == RS_FINAL;
        }
        ctl->all_done = all;
        ctl->all_conf = conf;
        ctl->any_rep = 0;
    }
}

// True residual from w64 = (K W^T W + sigma^2 I) x_hat (FP64):
//   r_hat = r_hat_0 - w64 (- c^x kg for GEN), with c^r = 1 - sigma^2 c^x
template <typename T, bool GEN>
__global__ void k_cg_resid(int64_t m, int R, const double *__restrict__ w64, const double *__restrict__ r0,
                           const T *__restrict__ kg, T *__restrict__ r, const double *__restrict__ S,
                           const int *__restrict__ state, const int *__restrict__ want, const CgCtl *__restrict__ ctl) {
    if (ctl->all_conf) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(e / m);
        if (state[rr] == RS_FINAL || !(want[rr] || state[rr] == RS_TENTATIVE)) continue;
        double v = r0[e] - w64[e];
        if (GEN) v -= S[F_CX * R + rr] * (double)kg[e];
        r[e] = (T)v;
    }
}

// ------------------------------------------------------------------ workspace
struct SolveWork {
    KgOp *kg[3];  // K_G operators by element type: FP32, FP64, double-float
    void *buf;
    size_t buf_bytes;
    double *S;
    double *part;
    int *state;
    int *want;
    int *iters;
    CgCtl *ctl;
    double *hist;     // alpha then beta, (maxiter + 1) x R each
    size_t hist_cap;  // entries per array
    int *hflag;       // pinned host: all_conf
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
    for (int i = 0; i < 3; ++i) kgop_destroy(w->kg[i]);
    if (w->buf) cudaFree(w->buf);
    if (w->S) cudaFree(w->S);
    if (w->part) cudaFree(w->part);
    if (w->state) cudaFree(w->state);
    if (w->want) cudaFree(w->want);
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
        FK_TRY(dev_alloc((void **)&w->state, sizeof(int) * MAX_R));
        FK_TRY(dev_alloc((void **)&w->want, sizeof(int) * MAX_R));
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
    const int i = dtype == FKSKI_F32 ? 0 : (dtype == FK_DF ? 2 : 1);
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

// Converted copies of the statistics in the solve precision.  Double-float solves read the FP32
// band (stored, or converted from FP64 statistics) and double-float copies of W^T y and W^T z.
template <typename T>
static int stats_as(fkski_stats *st, const BandT<T> **band, const T **wty, const T **wtz, cudaStream_t s) {
    if constexpr (std::is_same<T, dfl>::value) {
        const float *bf, *wf, *zf;
        FK_TRY(stats_as<float>(st, &bf, &wf, &zf, s));
        *band = bf;
        if (!st->wty_df) {
            FK_TRY(dev_alloc(&st->wty_df, sizeof(dfl) * st->m));
            k_convert<dfl><<<256, 256, 0, s>>>(st->wty, st->dtype == FKSKI_F64, (dfl *)st->wty_df, st->m);
            FK_LAUNCH();
            if (st->nprobes > 0) {
                FK_TRY(dev_alloc(&st->wtz_df, sizeof(dfl) * st->nprobes * st->m));
                k_convert<dfl><<<1024, 256, 0, s>>>(st->wtz, st->dtype == FKSKI_F64, (dfl *)st->wtz_df,
                                                    st->nprobes * st->m);
                FK_LAUNCH();
            }
        }
        *wty = (const dfl *)st->wty_df;
        *wtz = (const dfl *)st->wtz_df;
        return FKSKI_OK;
    } else {
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
}

int stats_band_as(fkski_stats *st, int dtype, const void **band, const void **wty, const void **wtz, cudaStream_t s) {
    if (dtype == FKSKI_F32) return stats_as<float>(st, (const float **)band, (const float **)wty, (const float **)wtz, s);
    if (dtype == FK_DF) return stats_as<dfl>(st, (const float **)band, (const dfl **)wty, (const dfl **)wtz, s);
    return stats_as<double>(st, (const double **)band, (const double **)wty, (const double **)wtz, s);
}

// Launch the captured iteration chunk (captured on w->ws) until every rhs is final, running the
// captured residual-replacement pass whenever a chunk leaves a request for it.  The internal
// stream first waits for the caller's stream, and the caller's stream waits for it at the end.
static size_t graph_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (!g || cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    size_t k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

static int run_graph_loop(cudaGraphExec_t body, cudaGraphExec_t rep, SolveWork *w, int maxiter, int check,
                          cudaStream_t s, long long nbody, long long nrep) {
    FK_CUDA(cudaEventRecord(w->ev, s));
    FK_CUDA(cudaStreamWaitEvent(w->ws, w->ev, 0));
    int launched = 0;
    while (launched <= maxiter + check) {
        FK_CUDA(cudaGraphLaunch(body, w->ws));
        count_launches(nbody);
        launched += check;
        FK_CUDA(cudaMemcpyAsync(w->hflag, &w->ctl->all_conf, 2 * sizeof(int), cudaMemcpyDeviceToHost, w->ws));
        FK_CUDA(cudaStreamSynchronize(w->ws));
        if (w->hflag[0]) break;
        if (rep && w->hflag[1]) {
            FK_CUDA(cudaGraphLaunch(rep, w->ws));
            count_launches(nrep);
            FK_CUDA(cudaMemcpyAsync(w->hflag, &w->ctl->all_conf, 2 * sizeof(int), cudaMemcpyDeviceToHost, w->ws));
            FK_CUDA(cudaStreamSynchronize(w->ws));
            if (w->hflag[0]) break;
        }
    }
    FK_CUDA(cudaEventRecord(w->ev, w->ws));
    FK_CUDA(cudaStreamWaitEvent(s, w->ev, 0));
    return FKSKI_OK;
}

template <typename T>
struct CgVecs {
    T *r, *p, *u, *v, *s, *z, *g, *kg, *g0;  // solve precision (g = W^T b', g0 = W^T b)
    double *x, *r0, *t64, *w64;              // FP64: solution, r_hat_0, temporaries
};

// ---- setup kernels for the compressed base vectors (GEN)
// few fixed CG steps on (W^T W) b_hat = W^T b (any b_hat gives an exact splitting b = W b_hat + b')
template <typename T>
__global__ void k_bcg_xr(int64_t m, int R, T *__restrict__ X, T *__restrict__ Rr, const T *__restrict__ P,
                         const T *__restrict__ Q, const double *__restrict__ sums, const double *__restrict__ rr,
                         const int *__restrict__ mask) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / m);
        const double pq = sums[r * 4];
        if (!mask[r] || !(pq > 0.0) || !(rr[r] > 0.0)) continue;
        const T a = (T)(rr[r] / pq);
        X[e] = fma(a, P[e], X[e]);
        Rr[e] = fma(-a, Q[e], Rr[e]);
    }
}

template <typename T>
__global__ void k_bcg_p(int64_t m, int R, T *__restrict__ P, const T *__restrict__ Rr, const double *__restrict__ sums,
                        const double *__restrict__ rr, const int *__restrict__ mask) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / m);
        if (!mask[r] || !(rr[r] > 0.0)) continue;
        const T be = (T)(sums[r * 4] / rr[r]);
        P[e] = fma(be, P[e], Rr[e]);
    }
}

// r0: rebased rows b_hat (from X), Alg. 5 rows -K_G W^T y / sigma^2 (from w64, already K applied)
template <typename T>
__global__ void k_r0_init(int64_t m, int R, const T *__restrict__ X, const double *__restrict__ kgy, double s2,
                          double *__restrict__ r0, T *__restrict__ r, const int *__restrict__ mask) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int rr = (int)(e / m);
        const double v = mask[rr] ? (double)X[e] : -kgy[e] / s2;
        r0[e] = v;
        r[e] = (T)v;
    }
}

// g' = W^T b' = W^T b - W^T W b_hat (rebased rows), 0 for Alg. 5 rows
template <typename T>
__global__ void k_gprime(int64_t m, int R, const T *__restrict__ g0, const double *__restrict__ Bb, T *__restrict__ gp,
                         const int *__restrict__ mask) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / m);
        gp[e] = mask[r] ? (T)((double)g0[e] - Bb[e]) : T(0);
    }
}

// sums[r*4+0] = b_hat . W^T b, sums[r*4+1] = b_hat . W^T W b_hat  (FP64)
__global__ void k_rebase_scalars(const double *__restrict__ sums, double *__restrict__ S, int R, double s2,
                                 const int *__restrict__ mask) {
    const int r = threadIdx.x;
    if (r >= R) return;
    if (mask[r]) {
        const double bg = sums[r * 4], bbb = sums[r * 4 + 1];
        S[F_RHOP * R + r] = fmax(S[F_RHO0 * R + r] - 2.0 * bg + bbb, 0.0);
        S[F_BG * R + r] = bg - bbb;
        S[F_C0 * R + r] = 0.0;
    } else {
        S[F_RHOP * R + r] = 0.0;
        S[F_BG * R + r] = 0.0;
        S[F_C0 * R + r] = 1.0 / s2;
    }
    S[F_CR * R + r] = 1.0;
    S[F_CP * R + r] = 1.0;
    S[F_CX * R + r] = 0.0;
}

constexpr int BCG_STEPS = 8;

// One factorized-CG solve of A x = b for R right-hand sides (b_0 = y, b_p = z_p).
// GEN = false: Alg. 5 on y (R = 1).  GEN = true: compressed form with per-rhs base vectors;
// rebase[r] = 1 splits b_r = W b_hat + b' (x0 = 0, the Lanczos start for SLQ), rebase[r] = 0 uses
// Alg. 5's start x0 = b / sigma^2 for that rhs.  On return V.x holds x_hat (FP64); the scalars and
// coefficient histories stay in the workspace.
// One factorized-CG solve split in phases, so that several independent problems can run their
// iteration chunks from one graph launch: prepare (set-up launches on the caller's stream and
// capture of the chunk graphs), the chunk loop, and collect (results to the host).
struct FcgGraphs {
    cudaGraph_t body = nullptr, rep = nullptr;
    long long nbody = 0, nrep = 0;
    int check = 1;
    void release() {
        if (body) cudaGraphDestroy(body);
        if (rep) cudaGraphDestroy(rep);
        body = rep = nullptr;
    }
};

// r0_in (optional, non-GEN only): right-hand sides b_r = W r0_in[r] in span(W) with x0 = 0 (the
// second start of App. B that puts r0 in span(W), e.g. posterior covariance); device FP64 R x m,
// with ||b_r||^2 in rho0_in (host).  Without it row 0 solves for y from x0 = y / sigma^2.
template <typename T, bool GEN>
static int fcg_prepare(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, int R, const int *rebase,
                       CgVecs<T> &V, FcgGraphs &G, cudaStream_t s, const double *r0_in = nullptr,
                       const double *rho0_in = nullptr) {
    if (r0_in && (GEN || !rho0_in)) return FKSKI_E_INVALID_ARG;
    SolveWork *w;
    FK_TRY(work_get(st, &w));
    const int dt = dtype_of<T>();
    KgOp *kg, *kg64;
    FK_TRY(work_kg(st, w, dt, &kg));
    FK_TRY(work_kg(st, w, FKSKI_F64, &kg64));
    FK_TRY(kgop_set(kg, kern, -1, s));
    if (kg64 != kg) FK_TRY(kgop_set(kg64, kern, -1, s));
    using TB = BandT<T>;
    const TB *band;
    const T *wty, *wtz;
    FK_TRY(stats_as<T>(st, &band, &wty, &wtz, s));
    const int64_t m = st->m;
    const size_t nT = (size_t)R * m;
    FK_TRY(work_buf(w, sizeof(T) * 9 * nT + sizeof(double) * 4 * nT + 256));
    T *b = (T *)w->buf;
    V.r = b; V.p = b + nT; V.u = b + 2 * nT; V.v = b + 3 * nT; V.s = b + 4 * nT; V.z = b + 5 * nT;
    V.g = b + 6 * nT; V.kg = b + 7 * nT; V.g0 = b + 8 * nT;
    double *d64 = (double *)((char *)w->buf + ((sizeof(T) * 9 * nT + 255) / 256) * 256);
    V.x = d64; V.r0 = d64 + nT; V.t64 = d64 + 2 * nT; V.w64 = d64 + 3 * nT;
    FK_TRY(work_hist(w, R, o->maxiter));
    double *ha = w->hist, *hb = w->hist + w->hist_cap;
    const double s2 = kern->noise_var;
    CgCtl hc;
    memset(&hc, 0, sizeof(hc));
    hc.maxiter = o->maxiter;
    hc.R = R;
    hc.sig2 = s2;
    // reliable updates: on for FP32 vectors unless the caller chose (1 on, 2 off); FP64 and
    // double-float recurrences track the true residual without them
    hc.replace = o->reliable_updates == 1 ? 1 : (o->reliable_updates == 2 ? 0 : (std::is_same<T, float>::value ? 1 : 0));
    hc.delta2 = 0.01;
    FK_CUDA(cudaMemcpyAsync(w->ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, s));
    std::vector<double> hS((size_t)NF * R, 0.0);
    for (int r = 0; r < R; ++r) {
        const double rho = r0_in ? rho0_in[r] : (r == 0 ? st->yty : st->ztz[r - 1]);
        hS[F_RHO0 * R + r] = rho;
        hS[F_EPS * R + r] = o->rtol * o->rtol * rho;
        hS[F_C0 * R + r] = r0_in ? 0.0 : 1.0 / s2;
    }
    FK_CUDA(cudaMemcpyAsync(w->S, hS.data(), sizeof(double) * NF * R, cudaMemcpyHostToDevice, s));
    FK_CUDA(cudaMemsetAsync(w->state, 0, sizeof(int) * R, s));
    FK_CUDA(cudaMemsetAsync(w->want, 0, sizeof(int) * R, s));
    FK_CUDA(cudaMemsetAsync(w->iters, 0, sizeof(int) * R, s));
    FK_CUDA(cudaMemsetAsync(b, 0, sizeof(T) * 8 * nT, s));
    FK_CUDA(cudaMemsetAsync(V.x, 0, sizeof(double) * nT, s));
    const unsigned gb = (unsigned)grid_blocks(m);
    const unsigned gv = (unsigned)std::min<int64_t>(cdiv((int64_t)nT, 256), 152 * 8);
    const double *sig2_dev = &w->ctl->sig2;
    const int *gate_done = &w->ctl->all_done;
    const int *gate_conf = &w->ctl->all_conf;
    const int NQ = GEN ? 2 : 1;
    if (r0_in) {
        FK_CUDA(cudaMemsetAsync(V.g0, 0, sizeof(T) * nT, s));  // x0 = 0: no W^T b term in W^T x
    } else {
        // W^T b for every rhs
        FK_CUDA(cudaMemcpyAsync(V.g0, wty, sizeof(T) * m, cudaMemcpyDeviceToDevice, s));
        if (R > 1) FK_CUDA(cudaMemcpyAsync(V.g0 + m, wtz, sizeof(T) * (R - 1) * m, cudaMemcpyDeviceToDevice, s));
        // K_G W^T b in FP64 (for the Alg. 5 starts)
        k_convert_t<T, double><<<gv, 256, 0, s>>>(V.g0, V.t64, (int64_t)nT, 1.0);
        FK_LAUNCH();
        FK_TRY(kgop_apply(kg64, V.t64, V.w64, R, nullptr, 0.0, s));
    }
    int *mask = w->want;  // reused below as the replacement flags (reset after setup)
    if (GEN) {
        std::vector<int> hm(R);
        for (int r = 0; r < R; ++r) hm[r] = rebase ? rebase[r] : 1;
        FK_CUDA(cudaMemcpyAsync(mask, hm.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
        // b_hat: BCG_STEPS CG steps on (W^T W) b_hat = W^T b; X = V.u, Rr = V.v, P = V.p, Q = V.s
        double *sums = V.r0;   // scratch (4 R doubles) until r0 is written
        double *rr = V.r0 + 4 * R;
        FK_CUDA(cudaMemcpyAsync(V.v, V.g0, sizeof(T) * nT, cudaMemcpyDeviceToDevice, s));
        FK_CUDA(cudaMemcpyAsync(V.p, V.g0, sizeof(T) * nT, cudaMemcpyDeviceToDevice, s));
        k_dots4<T, T><<<gb, CG_T, 0, s>>>(V.v, V.v, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, m, R, w->part, nullptr);
        k_fin_sums<<<(unsigned)cdiv(R * 4 * 32, 256), 256, 0, s>>>(w->part, gb, R, 4, sums);
        k_pick<<<1, 128, 0, s>>>(sums, 4, R, rr);
        FK_LAUNCH();
        for (int it = 0; it < BCG_STEPS; ++it) {
            FK_TRY((launch_spmv<TB, T>(band, st->grid, V.p, V.s, m, R, nullptr, 1, nullptr, nullptr, gb, s)));
            k_dots4<T, T><<<gb, CG_T, 0, s>>>(V.p, V.s, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, m, R, w->part, nullptr);
            k_fin_sums<<<(unsigned)cdiv(R * 4 * 32, 256), 256, 0, s>>>(w->part, gb, R, 4, sums);
            k_bcg_xr<T><<<gv, 256, 0, s>>>(m, R, V.u, V.v, V.p, V.s, sums, rr, mask);
            k_dots4<T, T><<<gb, CG_T, 0, s>>>(V.v, V.v, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, m, R, w->part, nullptr);
            k_fin_sums<<<(unsigned)cdiv(R * 4 * 32, 256), 256, 0, s>>>(w->part, gb, R, 4, sums);
            k_bcg_p<T><<<gv, 256, 0, s>>>(m, R, V.p, V.v, sums, rr, mask);
            k_pick<<<1, 128, 0, s>>>(sums, 4, R, rr);
            FK_LAUNCH();
        }
        // r_hat_0 (FP64 and T); W^T W b_hat in FP64; g' and the scalars of b'
        k_r0_init<T><<<gv, 256, 0, s>>>(m, R, V.u, V.w64, s2, V.r0, V.r, mask);
        FK_LAUNCH();
        FK_TRY((launch_spmv<TB, double>(band, st->grid, V.r0, V.t64, m, R, nullptr, 1, nullptr, nullptr, gb, s)));
        k_gprime<T><<<gv, 256, 0, s>>>(m, R, V.g0, V.t64, V.g, mask);
        k_convert_t<T, double><<<gv, 256, 0, s>>>(V.g0, V.w64, (int64_t)nT, 1.0);
        k_dots4<double, double><<<gb, CG_T, 0, s>>>(V.r0, V.w64, V.r0, V.t64, nullptr, nullptr, nullptr, nullptr, m, R,
                                                    w->part, nullptr);
        k_fin_sums<<<(unsigned)cdiv(R * 4 * 32, 256), 256, 0, s>>>(w->part, gb, R, 4, V.w64);
        k_rebase_scalars<<<1, 128, 0, s>>>(V.w64, w->S, R, s2, mask);
        FK_LAUNCH();
        FK_TRY(kgop_apply(kg, V.g, V.kg, R, nullptr, 0.0, s));
        k_dots4<T, T><<<gb, CG_T, 0, s>>>(V.g, V.kg, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, m, R, w->part, nullptr);
        k_fin_sums<<<(unsigned)cdiv(R * 4 * 32, 256), 256, 0, s>>>(w->part, gb, R, 4, V.w64);
        k_pick<<<1, 128, 0, s>>>(V.w64, 4, R, w->S + F_GKG * R);
        FK_LAUNCH();
        FK_CUDA(cudaMemsetAsync(mask, 0, sizeof(int) * R, s));
        FK_CUDA(cudaMemsetAsync(V.u, 0, sizeof(T) * 3 * nT, s));  // u, v, p back to zero (s below)
        FK_CUDA(cudaMemsetAsync(V.s, 0, sizeof(T) * nT, s));
    } else if (r0_in) {
        // b = W r0_in with x0 = 0: r = b, so r_hat_0 = r0_in
        FK_CUDA(cudaMemcpyAsync(V.r0, r0_in, sizeof(double) * nT, cudaMemcpyDeviceToDevice, s));
        k_convert_t<double, T><<<gv, 256, 0, s>>>(V.r0, V.r, (int64_t)nT, 1.0);
        FK_LAUNCH();
    } else {
        // r_hat_0 = -K_G W^T y / sigma^2 in FP64; r_hat = r_hat_0 in T
        k_convert_t<double, double><<<gv, 256, 0, s>>>(V.w64, V.r0, m, -1.0 / s2);
        FK_LAUNCH();
        k_convert_t<double, T><<<gv, 256, 0, s>>>(V.r0, V.r, m, 1.0);
        FK_LAUNCH();
    }
    // u = W^T W r with its partials, then the gamma step (taken by the product's last block when
    // the half-band kernel applies, else by its own one-block launch)
    auto spmv_gamma = [&](const int *gate, int mode, cudaStream_t st_) -> int {
        if constexpr (std::is_same<T, float>::value || std::is_same<T, dfl>::value) {
            if (R == 1) {
                const int rc0 = launch_spmvh_fin<GEN>(band, st->grid, V.r, V.u, m, w->part, NQ, GEN ? V.g : nullptr, gate,
                                                      (int)gb, CgFin{w->S, w->state, w->want, w->iters, hb, w->ctl, mode},
                                                      st_);
                if (rc0 != FKSKI_E_UNSUPPORTED) return rc0;
            }
        }
        FK_TRY((launch_spmv<TB, T>(band, st->grid, V.r, V.u, m, R, w->part, NQ, GEN ? V.g : nullptr, gate, gb, st_)));
        k_cg_fin_gamma<GEN><<<1, 256, 0, st_>>>(w->part, gb, w->S, w->state, w->want, w->iters, hb, w->ctl, mode);
        FK_LAUNCH();
        return FKSKI_OK;
    };
    // init pass: gamma_0, s_0 = u_0, z_0 = v_0, p_0 = r_0, alpha_0
    FK_TRY(spmv_gamma(nullptr, 1, s));
    FK_TRY(kgop_apply_dev(kg, V.u, V.v, R, V.r, sig2_dev, s));
    k_cg_psz<T, GEN><<<gb, CG_T, 0, s>>>(m, R, V.r, V.u, V.v, V.p, V.s, V.z, V.g, V.kg, w->part,
                                         CgFin{w->S, w->state, w->want, w->iters, ha, w->ctl, 1});
    FK_LAUNCH();
    FK_TRY(kgop_reserve(kg, R));
    FK_TRY(kgop_reserve(kg64, R));
    FK_TRY(kgop_tune(kg, R, s));
    if (hc.replace && kg64 != kg) FK_TRY(kgop_tune(kg64, R, s));
    // capture the iteration chunk, and (MIXED) the residual-replacement pass
    const int check = std::max(1, o->check_every);
    const cudaStream_t cs = w->ws;
    cudaGraph_t gbody = nullptr, grep = nullptr;
    const long long launches_before_capture = fkski_kernel_launches();
    FK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    int rc = FKSKI_OK;
    kgop_set_gate(kg, gate_done);  // finished solves skip their K_G passes too
    for (int it = 0; it < check && rc == FKSKI_OK; ++it) {
        k_cg_xr<T, GEN><<<gv, CG_T, 0, cs>>>(m, R, V.x, V.r, V.p, V.z, V.kg, w->S, w->state, w->ctl);
        rc = spmv_gamma(gate_done, 0, cs);
        if (rc) break;
        rc = kgop_apply_dev(kg, V.u, V.v, R, V.r, sig2_dev, cs);
        if (rc) break;
        k_cg_psz<T, GEN><<<gb, CG_T, 0, cs>>>(m, R, V.r, V.u, V.v, V.p, V.s, V.z, V.g, V.kg, w->part,
                                              CgFin{w->S, w->state, w->want, w->iters, ha, w->ctl, 0});
    }
    cudaError_t ce = cudaStreamEndCapture(cs, &gbody);
    kgop_set_gate(kg, nullptr);
    if (rc != FKSKI_OK) return rc;
    FK_CUDA(ce);
    if (hc.replace) {
        FK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        kgop_set_gate(kg64, gate_conf);
        // true residual in FP64: w64 = K (W^T W x_hat) + sigma^2 x_hat; gamma from it
        rc = launch_spmv<TB, double>(band, st->grid, V.x, V.t64, m, R, nullptr, 1, nullptr, gate_conf, gb, cs);
        if (rc == FKSKI_OK) rc = kgop_apply_dev(kg64, V.t64, V.w64, R, V.x, sig2_dev, cs);
        if (rc == FKSKI_OK) {
            k_cg_resid<T, GEN><<<gv, CG_T, 0, cs>>>(m, R, V.w64, V.r0, V.kg, V.r, w->S, w->state, w->want, w->ctl);
            rc = launch_spmv<TB, T>(band, st->grid, V.r, V.u, m, R, w->part, NQ, GEN ? V.g : nullptr, gate_conf, gb, cs);
        }
        if (rc == FKSKI_OK)
            k_cg_fin_replace<GEN><<<1, 256, 0, cs>>>(w->part, gb, w->S, w->state, w->want, w->iters, ha, w->ctl);
        ce = cudaStreamEndCapture(cs, &grep);
        kgop_set_gate(kg64, nullptr);
        if (rc != FKSKI_OK) { cudaGraphDestroy(gbody); return rc; }
        FK_CUDA(ce);
    }
    // captured launches are replays, counted when the graphs run
    count_launches(launches_before_capture - fkski_kernel_launches());
    G.body = gbody;
    G.rep = grep;
    G.nbody = (long long)graph_kernel_nodes(gbody);
    G.nrep = (long long)graph_kernel_nodes(grep);
    G.check = check;
    return FKSKI_OK;
}

// Iterations, residuals and status of a finished solve (synchronizes s).
template <typename T>
static int fcg_collect(fkski_stats *st, int R, int *iters_host, double *res_host, int *status_out, cudaStream_t s) {
    SolveWork *w = st->work;
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

template <typename T, bool GEN>
static int fcg_solve(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, int R, const int *rebase,
                     CgVecs<T> &V, int *iters_host, double *res_host, int *status_out, cudaStream_t s) {
    FcgGraphs G;
    FK_TRY((fcg_prepare<T, GEN>(st, kern, o, R, rebase, V, G, s)));
    cudaGraphExec_t ebody = nullptr, erep = nullptr;
    cudaError_t ce = cudaGraphInstantiate(&ebody, G.body, 0);
    if (ce == cudaSuccess && G.rep) ce = cudaGraphInstantiate(&erep, G.rep, 0);
    int rc = ce == cudaSuccess ? FKSKI_OK : note_cuda_error(ce, __FILE__, __LINE__);
    if (rc == FKSKI_OK) rc = run_graph_loop(ebody, erep, st->work, o->maxiter, G.check, s, G.nbody, G.nrep);
    if (ebody) cudaGraphExecDestroy(ebody);
    if (erep) cudaGraphExecDestroy(erep);
    G.release();
    if (rc) return rc;
    return fcg_collect<T>(st, R, iters_host, res_host, status_out, s);
}

// W^T x for each rhs in FP64: x = c0 b + W x_hat + c^x b'  ->  c0 W^T b + W^T W x_hat + c^x g
template <typename T>
__global__ void k_wtx64(const double *__restrict__ Bx, const T *__restrict__ g0, const T *__restrict__ gp,
                        double *__restrict__ out, int64_t m, int R, const double *__restrict__ S) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)R * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / m);
        out[e] = Bx[e] + S[F_C0 * R + r] * (double)g0[e] + S[F_CX * R + r] * (double)gp[e];
    }
}

template <typename T>
static int fcg_wtx64(fkski_stats *st, CgVecs<T> &V, int R, double *out64, cudaStream_t s) {
    SolveWork *w = st->work;
    const BandT<T> *band;
    const T *wty, *wtz;
    FK_TRY(stats_as<T>(st, &band, &wty, &wtz, s));
    const int64_t m = st->m;
    const unsigned gb = (unsigned)grid_blocks(m);
    const unsigned gv = (unsigned)std::min<int64_t>(cdiv((int64_t)R * m, 256), 152 * 8);
    FK_TRY((launch_spmv<BandT<T>, double>(band, st->grid, V.x, V.t64, m, R, nullptr, 1, nullptr, nullptr, gb, s)));
    k_wtx64<T><<<gv, 256, 0, s>>>(V.t64, V.g0, V.g, out64, m, R, w->S);
    FK_LAUNCH();
    return FKSKI_OK;
}

// a = W^T z (FP64 -> output type) and v = K_G a (FP64 product -> output type) of a finished
// single-rhs solve.
template <typename T>
static int mean_outputs(fkski_stats *st, CgVecs<T> &V, OutT<T> *a_out, OutT<T> *v_out, cudaStream_t s) {
    SolveWork *w = st->work;
    const int64_t m = st->m;
    FK_TRY(fcg_wtx64<T>(st, V, 1, V.w64, s));
    KgOp *kg64 = w->kg[1];
    FK_TRY(kgop_apply(kg64, V.w64, V.r0, 1, nullptr, 0.0, s));
    const unsigned gv = (unsigned)std::min<int64_t>(cdiv(m, 256), 152 * 8);
    k_convert_t<double, OutT<T>><<<gv, 256, 0, s>>>(V.w64, a_out, m, 1.0);
    FK_LAUNCH();
    k_convert_t<double, OutT<T>><<<gv, 256, 0, s>>>(V.r0, v_out, m, 1.0);
    FK_LAUNCH();
    return FKSKI_OK;
}

template <typename T>
static int solve_mean(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, bool gen, OutT<T> *a_out,
                      OutT<T> *v_out, fkski_info *info, cudaStream_t s) {
    CgVecs<T> V;
    int it = 0, status = 0;
    double res = 0.0;
    const int rebase = 1;
    if (gen) FK_TRY((fcg_solve<T, true>(st, kern, o, 1, &rebase, V, &it, &res, &status, s)));
    else FK_TRY((fcg_solve<T, false>(st, kern, o, 1, nullptr, V, &it, &res, &status, s)));
    FK_TRY(mean_outputs<T>(st, V, a_out, v_out, s));
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
    if (o.x0_mode != FKSKI_X0_ZERO && o.x0_mode != FKSKI_X0_Y_OVER_S2) return FKSKI_E_INVALID_ARG;
    if (info) memset(info, 0, sizeof(*info));
    const bool gen = o.x0_mode == FKSKI_X0_ZERO;
    if (o.precision == FKSKI_DOUBLE)
        return solve_mean<double>(st, kern, &o, gen, (double *)a_out, (double *)v_out, info, s);
    if (o.precision == FKSKI_FP32)
        return solve_mean<float>(st, kern, &o, gen, (float *)a_out, (float *)v_out, info, s);
    if (o.precision != FKSKI_MIXED) return FKSKI_E_INVALID_ARG;
    return solve_mean<dfl>(st, kern, &o, gen, (float *)a_out, (float *)v_out, info, s);
}

// ------------------------------------------------------------------ batch of independent problems
// Every problem is prepared as for fkski_solve (set-up launches, captured chunk graphs), then one
// parent graph holds all chunk graphs as independent child nodes (the GPU runs them
// concurrently) followed by one small kernel that gathers every problem's flags; each replay
// advances every unfinished problem by check_every iterations and costs one flag read.
__global__ void k_gather_flags(CgCtl *const *__restrict__ ctls, int P, int *__restrict__ flags) {
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        flags[2 * p] = ctls[p]->all_conf;
        flags[2 * p + 1] = ctls[p]->any_rep;
    }
}

static int parent_graph(const std::vector<cudaGraph_t> &kids, CgCtl **dctls, int P, int *dflags, cudaGraphExec_t *exec) {
    cudaGraph_t g = nullptr;
    FK_CUDA(cudaGraphCreate(&g, 0));
    std::vector<cudaGraphNode_t> nodes;
    int rc = FKSKI_OK;
    for (cudaGraph_t k : kids) {
        if (!k) continue;
        cudaGraphNode_t nd;
        const cudaError_t e = cudaGraphAddChildGraphNode(&nd, g, nullptr, 0, k);
        if (e != cudaSuccess) { rc = note_cuda_error(e, __FILE__, __LINE__); break; }
        nodes.push_back(nd);
    }
    if (rc == FKSKI_OK) {
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        void *args[] = {(void *)&dctls, (void *)&P, (void *)&dflags};
        kp.func = (void *)k_gather_flags;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(128);
        kp.kernelParams = args;
        cudaGraphNode_t nd;
        cudaError_t e = cudaGraphAddKernelNode(&nd, g, nodes.data(), nodes.size(), &kp);
        if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
        if (e != cudaSuccess) rc = note_cuda_error(e, __FILE__, __LINE__);
    }
    cudaGraphDestroy(g);
    return rc;
}

template <typename T>
static int solve_batched_typed(int P, fkski_stats *const *sts, const fkski_kernel *kernels, const fkski_opts *o,
                               void *const *a_out, void *const *v_out, fkski_info *info, cudaStream_t s) {
    const bool gen = o->x0_mode == FKSKI_X0_ZERO;
    std::vector<CgVecs<T>> V(P);
    std::vector<FcgGraphs> G(P);
    const int rebase = 1;
    int rc = FKSKI_OK;
    for (int p = 0; p < P && rc == FKSKI_OK; ++p)
        rc = gen ? fcg_prepare<T, true>(sts[p], &kernels[p], o, 1, &rebase, V[p], G[p], s)
                 : fcg_prepare<T, false>(sts[p], &kernels[p], o, 1, nullptr, V[p], G[p], s);
    CgCtl **dctls = nullptr;
    int *dflags = nullptr, *hflags = nullptr;
    cudaGraphExec_t eb = nullptr, er = nullptr;
    long long nb = 1, nr = 1;
    std::vector<cudaGraph_t> kb, kr;
    for (int p = 0; p < P; ++p) {
        kb.push_back(G[p].body);
        kr.push_back(G[p].rep);
        nb += G[p].nbody;
        nr += G[p].nrep;
    }
    const bool any_rep_graph = std::any_of(kr.begin(), kr.end(), [](cudaGraph_t g) { return g != nullptr; });
    if (rc == FKSKI_OK) {
        std::vector<CgCtl *> hctls(P);
        for (int p = 0; p < P; ++p) hctls[p] = sts[p]->work->ctl;
        cudaError_t e = pool_alloc((void **)&dctls, sizeof(CgCtl *) * P, s) == FKSKI_OK ? cudaSuccess : cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = pool_alloc((void **)&dflags, sizeof(int) * 2 * P, s) == FKSKI_OK ? cudaSuccess : cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaMemcpyAsync(dctls, hctls.data(), sizeof(CgCtl *) * P, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&hflags, sizeof(int) * 2 * P);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // hctls is a host temporary
        if (e != cudaSuccess) rc = note_cuda_error(e, __FILE__, __LINE__);
    }
    if (rc == FKSKI_OK) rc = parent_graph(kb, dctls, P, dflags, &eb);
    if (rc == FKSKI_OK && any_rep_graph) rc = parent_graph(kr, dctls, P, dflags, &er);
    for (auto &g : G) g.release();
    if (rc == FKSKI_OK) {
        SolveWork *w0 = sts[0]->work;
        const cudaStream_t ws = w0->ws;
        const int check = G[0].check;
        cudaError_t e = cudaEventRecord(w0->ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ws, w0->ev, 0);
        int launched = 0;
        while (e == cudaSuccess && launched <= o->maxiter + check) {
            e = cudaGraphLaunch(eb, ws);
            count_launches(nb);
            launched += check;
            if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, dflags, sizeof(int) * 2 * P, cudaMemcpyDeviceToHost, ws);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ws);
            if (e != cudaSuccess) break;
            bool all = true, rep = false;
            for (int p = 0; p < P; ++p) {
                all = all && hflags[2 * p];
                rep = rep || hflags[2 * p + 1];
            }
            if (all) break;
            if (er && rep) {
                e = cudaGraphLaunch(er, ws);
                count_launches(nr);
                if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, dflags, sizeof(int) * 2 * P, cudaMemcpyDeviceToHost, ws);
                if (e == cudaSuccess) e = cudaStreamSynchronize(ws);
                if (e != cudaSuccess) break;
                all = true;
                for (int p = 0; p < P; ++p) all = all && hflags[2 * p];
                if (all) break;
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(w0->ev, ws);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, w0->ev, 0);
        if (e != cudaSuccess) rc = note_cuda_error(e, __FILE__, __LINE__);
    }
    if (eb) cudaGraphExecDestroy(eb);
    if (er) cudaGraphExecDestroy(er);
    int worst = FKSKI_OK;
    for (int p = 0; p < P && rc == FKSKI_OK; ++p) {
        int it = 0, status = FKSKI_OK;
        double res = 0.0;
        rc = fcg_collect<T>(sts[p], 1, &it, &res, &status, s);
        if (rc == FKSKI_OK) rc = mean_outputs<T>(sts[p], V[p], (OutT<T> *)a_out[p], (OutT<T> *)v_out[p], s);
        if (info) {
            info[p].iters = it;
            info[p].iters_rhs[0] = it;
            info[p].rel_residual = res;
            info[p].status = status;
        }
        if (status == FKSKI_E_BREAKDOWN || (status != FKSKI_OK && worst == FKSKI_OK)) worst = status;
    }
    if (dctls) cudaFreeAsync(dctls, s);
    if (dflags) cudaFreeAsync(dflags, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (hflags) cudaFreeHost(hflags);
    if (rc == FKSKI_OK && e != cudaSuccess) rc = note_cuda_error(e, __FILE__, __LINE__);
    return rc != FKSKI_OK ? rc : worst;
}

int solve_batched_impl(int P, fkski_stats *const *sts, const fkski_kernel *kernels, const fkski_opts *opts,
                       void *const *a_out, void *const *v_out, fkski_info *info, cudaStream_t s) {
    if (P < 1 || !sts || !kernels || !a_out || !v_out) return FKSKI_E_INVALID_ARG;
    fkski_opts o;
    if (opts) o = *opts; else fkski_default_opts(&o);
    if (o.maxiter < 1 || !(o.rtol >= 0.0)) return FKSKI_E_INVALID_ARG;
    if (o.x0_mode != FKSKI_X0_ZERO && o.x0_mode != FKSKI_X0_Y_OVER_S2) return FKSKI_E_INVALID_ARG;
    for (int p = 0; p < P; ++p) {
        if (!sts[p] || !a_out[p] || !v_out[p]) return FKSKI_E_INVALID_ARG;
        if (!(kernels[p].noise_var > 0.0) || !std::isfinite(kernels[p].noise_var)) return FKSKI_E_INVALID_ARG;
        for (int q = 0; q < p; ++q)
            if (sts[q] == sts[p]) return FKSKI_E_INVALID_ARG;  // one workspace per statistics object
    }
    if (info) memset(info, 0, sizeof(fkski_info) * P);
    if (o.precision == FKSKI_DOUBLE) return solve_batched_typed<double>(P, sts, kernels, &o, a_out, v_out, info, s);
    if (o.precision == FKSKI_FP32) return solve_batched_typed<float>(P, sts, kernels, &o, a_out, v_out, info, s);
    if (o.precision != FKSKI_MIXED) return FKSKI_E_INVALID_ARG;
    return solve_batched_typed<dfl>(P, sts, kernels, &o, a_out, v_out, info, s);
}

int band_mvm_impl(const fkski_stats *stc, const void *x, void *u, int nrhs, int dtype, cudaStream_t s) {
    if (!stc || !x || !u || nrhs < 1) return FKSKI_E_INVALID_ARG;
    fkski_stats *st = const_cast<fkski_stats *>(stc);
    const unsigned gb = (unsigned)grid_blocks(st->m);
    if (dtype == FKSKI_F32) {
        const float *band, *wty, *wtz;
        FK_TRY(stats_as<float>(st, &band, &wty, &wtz, s));
        return launch_spmv<float, float>(band, st->grid, (const float *)x, (float *)u, st->m, nrhs, nullptr, 1, nullptr,
                                         nullptr, gb, s);
    }
    if (dtype == FK_DF) {
        const float *band;
        const dfl *wty, *wtz;
        FK_TRY(stats_as<dfl>(st, &band, &wty, &wtz, s));
        return launch_spmv<float, dfl>(band, st->grid, (const dfl *)x, (dfl *)u, st->m, nrhs, nullptr, 1, nullptr,
                                       nullptr, gb, s);
    }
    if (dtype != FKSKI_F64) return FKSKI_E_INVALID_ARG;
    // FP64 vectors against the stored band (FP32 values promoted when the statistics are FP32)
    if (st->dtype == FKSKI_F32)
        return launch_spmv<float, double>((const float *)st->band, st->grid, (const double *)x, (double *)u, st->m, nrhs,
                                          nullptr, 1, nullptr, nullptr, gb, s);
    return launch_spmv<double, double>((const double *)st->band, st->grid, (const double *)x, (double *)u, st->m, nrhs,
                                       nullptr, 1, nullptr, nullptr, gb, s);
}

// ------------------------------------------------------------------ log-likelihood solves
// One batched solve of [y, z_1..z_T]: y starts from x0 = y / sigma^2 (Alg. 5's start, no
// rebasing needed), each probe from x0 = 0 with the rebased compressed form (its CG coefficients
// are those of the Krylov space of z_p, as SLQ needs).  Outputs for the gradient:
//   sol[r] = W^T x_r (solve precision, R x m), a64 = W^T x_0 (FP64, m),
//   zx[r] = b_r^T x_r = c0 rho0 + (W^T b).x_hat + c^x (b_hat . W^T b' + ||b'||^2)  (FP64, device).
__global__ void k_zx(const double *__restrict__ sums, const double *__restrict__ S, int R, double *__restrict__ zx) {
    const int r = threadIdx.x;
    if (r < R)
        zx[r] = S[F_C0 * R + r] * S[F_RHO0 * R + r] + sums[r * 4] +
                S[F_CX * R + r] * (S[F_BG * R + r] + S[F_RHOP * R + r]);
}

template <typename T>
static int grad_solve_t(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, T *sol, double *a64, double *zx,
                        int *iters, double *res, int *status, cudaStream_t s) {
    const int R = 1 + st->nprobes;
    CgVecs<T> V;
    std::vector<int> rebase(R, 1);
    rebase[0] = 0;
    FK_TRY((fcg_solve<T, true>(st, kern, o, R, rebase.data(), V, iters, res, status, s)));
    SolveWork *w = st->work;
    const int64_t m = st->m;
    FK_TRY(fcg_wtx64<T>(st, V, R, V.w64, s));
    const unsigned gv = (unsigned)std::min<int64_t>(cdiv((int64_t)R * m, 256), 152 * 8);
    k_convert_t<double, T><<<gv, 256, 0, s>>>(V.w64, sol, (int64_t)R * m, 1.0);
    FK_LAUNCH();
    FK_CUDA(cudaMemcpyAsync(a64, V.w64, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    const unsigned gb = (unsigned)grid_blocks(m);
    k_dots4<T, double><<<gb, CG_T, 0, s>>>(V.g0, V.x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, m, R, w->part,
                                           nullptr);
    FK_LAUNCH();
    k_fin_sums<<<(unsigned)cdiv(R * 4 * 32, 256), 256, 0, s>>>(w->part, gb, R, 4, V.t64);
    FK_LAUNCH();
    k_zx<<<1, 128, 0, s>>>(V.t64, w->S, R, zx);
    FK_LAUNCH();
    return FKSKI_OK;
}

int grad_solve(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, int dtype, void *sol, double *a64,
               double *zx, int *iters, double *res, int *status, cudaStream_t s) {
    if (dtype == FKSKI_F32) return grad_solve_t<float>(st, kern, o, (float *)sol, a64, zx, iters, res, status, s);
    if (dtype == FK_DF) return grad_solve_t<dfl>(st, kern, o, (dfl *)sol, a64, zx, iters, res, status, s);
    return grad_solve_t<double>(st, kern, o, (double *)sol, a64, zx, iters, res, status, s);
}

// ------------------------------------------------------------------ predict
// mu(x*) = sum over the 4^d stencil nodes of w(x*) v  (Def. 1 / Fact 2 mean)
template <typename TX, typename TV, int D>
__device__ __forceinline__ TV predict_point(const TX *__restrict__ Xs, int64_t ns, int64_t i, const KeyParams &kp,
                                            const TV *__restrict__ v, int64_t s1, int64_t s2, int &bad) {
    int c[3] = {1, 1, 1};
    TX t[3] = {TX(0), TX(0), TX(0)};
    int st = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) st |= axis_cell<TX>(Xs[(int64_t)k * ns + i], kp, k, c[k], t[k]);
    if (st) {
        bad |= (st & 2) ? ST_NONFINITE : ST_OUT_OF_GRID;
        return TV(0);
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
    return acc;
}

template <typename TX, typename TV, int D>
__global__ void k_predict(const TX *__restrict__ Xs, int64_t ns, KeyParams kp, const TV *__restrict__ v,
                          TV *__restrict__ mu, int *__restrict__ status, int64_t s1, int64_t s2) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x)
        mu[i] = predict_point<TX, TV, D>(Xs, ns, i, kp, v, s1, s2, bad);
    if (bad) atomicOr(status, bad);
}

// Batch of independent problems with the same d: one launch over the concatenated test points;
// a thread finds its problem by binary search over the jobs' first indices.
template <typename TX, typename TV>
struct PredJob {
    KeyParams kp;
    const TX *Xs;
    const TV *v;
    TV *mu;
    int64_t ns, s1, s2, first;
};

template <typename TX, typename TV, int D>
__global__ void k_predict_batched(const PredJob<TX, TV> *__restrict__ jobs, int nj, int64_t total, int *__restrict__ status) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].first <= g) lo = mid; else hi = mid - 1;
        }
        const PredJob<TX, TV> &J = jobs[lo];
        int bad = 0;
        const int64_t i = g - J.first;
        J.mu[i] = predict_point<TX, TV, D>(J.Xs, J.ns, i, J.kp, J.v, J.s1, J.s2, bad);
        if (bad) atomicOr(&status[lo], bad);
    }
}

template <typename TX, typename TV>
static int predict_typed(const fkski_stats *st, const TV *v, const TX *Xs, int64_t ns, TV *mu, cudaStream_t s) {
    const KeyParams kp = make_key_params(st->grid);
    int *dst;
    FK_TRY(pool_alloc((void **)&dst, sizeof(int), s));
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


template <typename TX, typename TV>
static int predict_batched_typed(int P, const fkski_stats *const *st, const void *const *v, const void *const *Xs,
                                 const int64_t *ns, void *const *mu, int *status_out, cudaStream_t s) {
    std::vector<PredJob<TX, TV>> jobs[3];
    std::vector<int> owner[3];
    int64_t total[3] = {0, 0, 0};
    for (int p = 0; p < P; ++p) {
        if (ns[p] == 0) continue;
        const int d = st[p]->d;
        PredJob<TX, TV> J;
        memset(&J, 0, sizeof(J));
        J.kp = make_key_params(st[p]->grid);
        J.Xs = (const TX *)Xs[p];
        J.v = (const TV *)v[p];
        J.mu = (TV *)mu[p];
        J.ns = ns[p];
        const int64_t M1 = st[p]->grid.M[1], M2 = st[p]->grid.M[2];
        J.s1 = d == 2 ? M1 : M1 * M2;
        J.s2 = M2;
        J.first = total[d - 1];
        total[d - 1] += ns[p];
        jobs[d - 1].push_back(J);
        owner[d - 1].push_back(p);
    }
    size_t jb = 0;
    for (int k = 0; k < 3; ++k) jb += jobs[k].size();
    PredJob<TX, TV> *dj = nullptr;
    int *dst = nullptr;
    FK_TRY(pool_alloc((void **)&dj, sizeof(PredJob<TX, TV>) * std::max<size_t>(jb, 1), s));
    FK_TRY(pool_alloc((void **)&dst, sizeof(int) * std::max<size_t>(jb, 1), s));
    FK_CUDA(cudaMemsetAsync(dst, 0, sizeof(int) * std::max<size_t>(jb, 1), s));
    std::vector<PredJob<TX, TV>> all;
    for (int k = 0; k < 3; ++k) all.insert(all.end(), jobs[k].begin(), jobs[k].end());
    if (jb) FK_CUDA(cudaMemcpyAsync(dj, all.data(), sizeof(PredJob<TX, TV>) * jb, cudaMemcpyHostToDevice, s));
    size_t off = 0;
    for (int k = 0; k < 3; ++k) {
        const int nj = (int)jobs[k].size();
        if (nj == 0) continue;
        const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total[k], 256), 152 * 16));
        if (k == 0) k_predict_batched<TX, TV, 1><<<gb, 256, 0, s>>>(dj + off, nj, total[k], dst + off);
        else if (k == 1) k_predict_batched<TX, TV, 2><<<gb, 256, 0, s>>>(dj + off, nj, total[k], dst + off);
        else k_predict_batched<TX, TV, 3><<<gb, 256, 0, s>>>(dj + off, nj, total[k], dst + off);
        FK_LAUNCH();
        off += nj;
    }
    std::vector<int> h(std::max<size_t>(jb, 1), 0);
    FK_CUDA(cudaMemcpyAsync(h.data(), dst, sizeof(int) * std::max<size_t>(jb, 1), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaFreeAsync(dj, s));
    FK_CUDA(cudaFreeAsync(dst, s));
    FK_CUDA(cudaStreamSynchronize(s));
    int worst = FKSKI_OK;
    off = 0;
    for (int p = 0; p < P; ++p) status_out[p] = FKSKI_OK;
    for (int k = 0; k < 3; ++k)
        for (size_t j = 0; j < jobs[k].size(); ++j, ++off) {
            const int rc = status_from_bits(h[off]);
            status_out[owner[k][j]] = rc;
            if (rc != FKSKI_OK && worst == FKSKI_OK) worst = rc;
        }
    return worst;
}

int predict_batched_impl(int P, const fkski_stats *const *st, const void *const *v, int vdtype, const void *const *Xs,
                         int xdtype, const int64_t *ns, void *const *mu, int *status, cudaStream_t s) {
    if (P < 1 || !st || !v || !Xs || !ns || !mu) return FKSKI_E_INVALID_ARG;
    for (int p = 0; p < P; ++p)
        if (!st[p] || ns[p] < 0 || (ns[p] > 0 && (!v[p] || !Xs[p] || !mu[p]))) return FKSKI_E_INVALID_ARG;
    std::vector<int> tmp(P);
    int *so = status ? status : tmp.data();
    if (vdtype == FKSKI_F32 && xdtype == FKSKI_F32) return predict_batched_typed<float, float>(P, st, v, Xs, ns, mu, so, s);
    if (vdtype == FKSKI_F64 && xdtype == FKSKI_F32) return predict_batched_typed<float, double>(P, st, v, Xs, ns, mu, so, s);
    if (vdtype == FKSKI_F32 && xdtype == FKSKI_F64) return predict_batched_typed<double, float>(P, st, v, Xs, ns, mu, so, s);
    if (vdtype == FKSKI_F64 && xdtype == FKSKI_F64) return predict_batched_typed<double, double>(P, st, v, Xs, ns, mu, so, s);
    return FKSKI_E_INVALID_ARG;
}

// ------------------------------------------------------------------ posterior covariance
// Exact SKI / GSGP posterior covariance at test points (Theorem 1, Claim 6):
//   cov(x_i, x_j) = w_i^T K w_j - (W K w_i)^T A^{-1} (W K w_j),  A = W K W^T + sigma^2 I
//                 = w_i^T c_j,   c_j = K w_j - K W^T A^{-1} W (K w_j).
// The right-hand side W (K w_j) lies in span(W), so each solve is the simplified EFCG from
// x0 = 0 with r_hat_0 = K w_j (App. B, second start), which returns W^T x = W^T W x_hat.
// Test points are solved in blocks of COV_R right-hand sides sharing one band read per
// iteration; c_j is gathered at all test points with the prediction weights.
constexpr int COV_R = 32;

// e[r] = w_{j0 + r} scattered on the grid (FP64); a point off the grid scatters nothing.
template <typename TX, int D>
__global__ void k_scatter_w(const TX *__restrict__ Xs, int64_t ns, int64_t j0, int R, KeyParams kp,
                            double *__restrict__ e, int64_t m, int64_t s1, int64_t s2, int *__restrict__ status) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int64_t i = j0 + r;
    int c[3] = {1, 1, 1};
    TX t[3] = {TX(0), TX(0), TX(0)};
    int st = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) st |= axis_cell<TX>(Xs[(int64_t)k * ns + i], kp, k, c[k], t[k]);
    if (st) {
        atomicOr(status, (st & 2) ? ST_NONFINITE : ST_OUT_OF_GRID);
        return;
    }
    double w[3][4];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        TX wx[4];
        keys_weights<TX>(t[k], wx);
#pragma unroll
        for (int a = 0; a < 4; ++a) w[k][a] = (double)wx[a];
    }
    double *er = e + (int64_t)r * m;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < (D > 1 ? 4 : 1); ++b)
            for (int q = 0; q < (D > 2 ? 4 : 1); ++q) {
                int64_t idx;
                double v;
                if (D == 1) { idx = c[0] - 1 + a; v = w[0][a]; }
                else if (D == 2) { idx = (int64_t)(c[0] - 1 + a) * s1 + (c[1] - 1 + b); v = w[0][a] * w[1][b]; }
                else {
                    idx = (int64_t)(c[0] - 1 + a) * s1 + (int64_t)(c[1] - 1 + b) * s2 + (c[2] - 1 + q);
                    v = w[0][a] * w[1][b] * w[2][q];
                }
                er[idx] = v;
            }
}

// cov[i][j0 + r] = w_i^T c_r for all test points i (row-major ns x ns, FP64)
template <typename TX, int D>
__global__ void k_cov_gather(const TX *__restrict__ Xs, int64_t ns, KeyParams kp, const double *__restrict__ C, int R,
                             int64_t m, int64_t j0, double *__restrict__ cov, int64_t s1, int64_t s2) {
    const int64_t total = ns * (int64_t)R;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % R);
        const int64_t i = e / R;
        int bad = 0;
        cov[i * ns + j0 + r] = predict_point<TX, double, D>(Xs, ns, i, kp, C + (int64_t)r * m, s1, s2, bad);
    }
}

__global__ void k_sub64(double *__restrict__ a, const double *__restrict__ b, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) a[e] -= b[e];
}

template <typename T, typename TX>
static int posterior_cov_typed(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, const TX *Xs, int64_t ns,
                               double *cov, fkski_info *info, cudaStream_t s) {
    const int64_t m = st->m;
    const int d = st->d;
    const KeyParams kp = make_key_params(st->grid);
    const int64_t M1 = st->grid.M[1], M2 = st->grid.M[2];
    const int64_t s1 = d == 2 ? M1 : M1 * M2, s2 = M2;
    SolveWork *w;
    FK_TRY(work_get(st, &w));
    KgOp *kg64;
    FK_TRY(work_kg(st, w, FKSKI_F64, &kg64));
    const BandT<T> *band;
    const T *wty, *wtz;
    FK_TRY(stats_as<T>(st, &band, &wty, &wtz, s));
    double *bh = nullptr, *tmp = nullptr, *sums = nullptr;
    int *dstatus = nullptr;
    const size_t nR = (size_t)COV_R * m;
    FK_TRY(pool_alloc((void **)&bh, sizeof(double) * nR, s));
    FK_TRY(pool_alloc((void **)&tmp, sizeof(double) * nR, s));
    FK_TRY(pool_alloc((void **)&sums, sizeof(double) * 4 * COV_R, s));
    FK_TRY(pool_alloc((void **)&dstatus, sizeof(int), s));
    FK_CUDA(cudaMemsetAsync(dstatus, 0, sizeof(int), s));
    const unsigned gb = (unsigned)grid_blocks(m);
    int rc = FKSKI_OK, worst = FKSKI_OK, itmax = 0;
    double resmax = 0.0;
    for (int64_t j0 = 0; j0 < ns && rc == FKSKI_OK; j0 += COV_R) {
        const int R = (int)std::min<int64_t>(COV_R, ns - j0);
        const int64_t nT = (int64_t)R * m;
        const unsigned gv = (unsigned)std::min<int64_t>(cdiv(nT, 256), 152 * 8);
        // b_hat_r = K w_r
        FK_CUDA(cudaMemsetAsync(tmp, 0, sizeof(double) * nT, s));
        if (d == 1) k_scatter_w<TX, 1><<<(R + 63) / 64, 64, 0, s>>>(Xs, ns, j0, R, kp, tmp, m, s1, s2, dstatus);
        else if (d == 2) k_scatter_w<TX, 2><<<(R + 63) / 64, 64, 0, s>>>(Xs, ns, j0, R, kp, tmp, m, s1, s2, dstatus);
        else k_scatter_w<TX, 3><<<(R + 63) / 64, 64, 0, s>>>(Xs, ns, j0, R, kp, tmp, m, s1, s2, dstatus);
        FK_LAUNCH();
        FK_TRY(kgop_set(kg64, kern, -1, s));
        FK_TRY(kgop_apply(kg64, tmp, bh, R, nullptr, 0.0, s));
        // ||W b_hat_r||^2 = b_hat_r^T (W^T W) b_hat_r
        FK_TRY((launch_spmv<BandT<T>, double>(band, st->grid, bh, tmp, m, R, nullptr, 1, nullptr, nullptr, gb, s)));
        k_dots4<double, double><<<gb, CG_T, 0, s>>>(bh, tmp, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, m, R,
                                                    w->part, nullptr);
        k_fin_sums<<<(unsigned)cdiv(R * 4 * 32, 256), 256, 0, s>>>(w->part, gb, R, 4, sums);
        FK_LAUNCH();
        std::vector<double> hs(4 * R), rho(R);
        FK_CUDA(cudaMemcpyAsync(hs.data(), sums, sizeof(double) * 4 * R, cudaMemcpyDeviceToHost, s));
        FK_CUDA(cudaStreamSynchronize(s));
        for (int r = 0; r < R; ++r) rho[r] = std::max(hs[4 * r], 1e-300);
        // solve A x_r = W b_hat_r from x0 = 0
        CgVecs<T> V;
        FcgGraphs G;
        rc = fcg_prepare<T, false>(st, kern, o, R, nullptr, V, G, s, bh, rho.data());
        cudaGraphExec_t eb = nullptr, er = nullptr;
        if (rc == FKSKI_OK) {
            cudaError_t e = cudaGraphInstantiate(&eb, G.body, 0);
            if (e == cudaSuccess && G.rep) e = cudaGraphInstantiate(&er, G.rep, 0);
            if (e != cudaSuccess) rc = note_cuda_error(e, __FILE__, __LINE__);
        }
        if (rc == FKSKI_OK) rc = run_graph_loop(eb, er, w, o->maxiter, G.check, s, G.nbody, G.nrep);
        if (eb) cudaGraphExecDestroy(eb);
        if (er) cudaGraphExecDestroy(er);
        G.release();
        std::vector<int> its(R);
        std::vector<double> res(R);
        int status = FKSKI_OK;
        if (rc == FKSKI_OK) rc = fcg_collect<T>(st, R, its.data(), res.data(), &status, s);
        if (rc != FKSKI_OK) break;
        for (int r = 0; r < R; ++r) {
            itmax = std::max(itmax, its[r]);
            resmax = std::max(resmax, res[r]);
        }
        if (status == FKSKI_E_BREAKDOWN || (status != FKSKI_OK && worst == FKSKI_OK)) worst = status;
        // c_r = b_hat_r - K W^T x_r  (W^T x_r = W^T W x_hat_r, FP64)
        FK_TRY(fcg_wtx64<T>(st, V, R, V.w64, s));
        FK_TRY(kgop_set(kg64, kern, -1, s));
        FK_TRY(kgop_apply(kg64, V.w64, tmp, R, nullptr, 0.0, s));
        k_sub64<<<gv, 256, 0, s>>>(bh, tmp, nT);
        FK_LAUNCH();
        const unsigned gg = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(ns * R, 256), 152 * 16));
        if (d == 1) k_cov_gather<TX, 1><<<gg, 256, 0, s>>>(Xs, ns, kp, bh, R, m, j0, cov, s1, s2);
        else if (d == 2) k_cov_gather<TX, 2><<<gg, 256, 0, s>>>(Xs, ns, kp, bh, R, m, j0, cov, s1, s2);
        else k_cov_gather<TX, 3><<<gg, 256, 0, s>>>(Xs, ns, kp, bh, R, m, j0, cov, s1, s2);
        FK_LAUNCH();
    }
    int hst = 0;
    FK_CUDA(cudaMemcpyAsync(&hst, dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(bh, s);
    cudaFreeAsync(tmp, s);
    cudaFreeAsync(sums, s);
    cudaFreeAsync(dstatus, s);
    FK_CUDA(cudaStreamSynchronize(s));
    if (info) {
        info->iters = itmax;
        info->rel_residual = resmax;
        info->status = worst;
    }
    if (rc != FKSKI_OK) return rc;
    const int pst = status_from_bits(hst);
    return pst != FKSKI_OK ? pst : worst;
}

int posterior_cov_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, const void *Xs, int xdtype,
                       int64_t ns, double *cov, fkski_info *info, cudaStream_t s) {
    if (!st || !kern || !Xs || !cov || ns < 1) return FKSKI_E_INVALID_ARG;
    fkski_opts o;
    if (opts) o = *opts; else fkski_default_opts(&o);
    if (!(kern->noise_var > 0.0) || !std::isfinite(kern->noise_var)) return FKSKI_E_INVALID_ARG;
    if (o.maxiter < 1 || !(o.rtol >= 0.0)) return FKSKI_E_INVALID_ARG;
    if (info) memset(info, 0, sizeof(*info));
    if (o.precision != FKSKI_MIXED && o.precision != FKSKI_DOUBLE && o.precision != FKSKI_FP32)
        return FKSKI_E_INVALID_ARG;
    if (xdtype == FKSKI_F32) {
        const float *X = (const float *)Xs;
        if (o.precision == FKSKI_DOUBLE) return posterior_cov_typed<double, float>(st, kern, &o, X, ns, cov, info, s);
        if (o.precision == FKSKI_FP32) return posterior_cov_typed<float, float>(st, kern, &o, X, ns, cov, info, s);
        return posterior_cov_typed<dfl, float>(st, kern, &o, X, ns, cov, info, s);
    }
    if (xdtype == FKSKI_F64) {
        const double *X = (const double *)Xs;
        if (o.precision == FKSKI_DOUBLE) return posterior_cov_typed<double, double>(st, kern, &o, X, ns, cov, info, s);
        if (o.precision == FKSKI_FP32) return posterior_cov_typed<float, double>(st, kern, &o, X, ns, cov, info, s);
        return posterior_cov_typed<dfl, double>(st, kern, &o, X, ns, cov, info, s);
    }
    return FKSKI_E_INVALID_ARG;
}

// ------------------------------------------------------------------ rank-k covariance (EFLA)
// Efficiently factorized Lanczos (App. B, EFLA; garbles read as in the oracle) on
// A = W K W^T + sigma^2 I started at b = y / ||y||, in FP64 with full reorthogonalisation.
// Lanczos vectors are kept compressed, q_i = W q_hat_i + d_i b, with P_hat_i = W^T W q_hat_i and
// s_hat_i = (K W^T W + sigma^2 I) q_hat_i, so one B(x) and no product with W per step.  Then
//   Q^T (W K w_x) = (P_hat + W^T b d^T)^T K w_x = G^T w_x,  G = K (P_hat + W^T b d^T),
// and with T = L L^T the predictive covariance is approximated (ref. [ConstantTimePD]) as
//   cov(x, x') ~ w_x^T K w_x' - (R^T w_x)^T (R^T w_x'),  R = G L^{-T}  (m x k, kept in st).
__global__ void k_efla_next(double *__restrict__ qn, const double *__restrict__ sh, const double *__restrict__ kwb,
                            const double *__restrict__ qprev, double c, double beta, int64_t m) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        qn[e] = sh[e] + c * kwb[e] - beta * qprev[e];
}

__global__ void k_axpy_d(double *__restrict__ y, const double *__restrict__ x, double a, int64_t m) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = fma(a, x[e], y[e]);
}

__global__ void k_scale_d(double *__restrict__ y, double a, int64_t m) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) y[e] *= a;
}

// out[j] = A[:, j] . v for the ncol columns of A (column stride m); one block per column.
__global__ void __launch_bounds__(256) k_gemv_t(const double *__restrict__ A, int ncol, int64_t m,
                                                 const double *__restrict__ v, double *__restrict__ out) {
    __shared__ double sh[8];
    const int j = blockIdx.x;
    if (j >= ncol) return;
    const double *a = A + (int64_t)j * m;
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < m; e += blockDim.x) acc = fma(a[e], v[e], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        out[j] = t;
    }
}

// v -= A[:, 0:ncol] c (column stride m), fixed summation order per element
__global__ void k_gemv_sub(const double *__restrict__ A, int ncol, int64_t m, const double *__restrict__ c,
                           double *__restrict__ v) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < ncol; ++j) acc = fma(A[(int64_t)j * m + e], c[j], acc);
        v[e] -= acc;
    }
}

// R[e][j] = sum_l G[l][e] Linvt[l][j] (G column-major m x k, R row-major m x k)
__global__ void k_lowrank_R(const double *__restrict__ G, const double *__restrict__ Linvt, int k, int64_t m,
                            double *__restrict__ R) {
    const int64_t total = m * (int64_t)k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / k;
        const int j = (int)(t % k);
        double acc = 0.0;
        for (int l = 0; l <= j; ++l) acc = fma(G[(int64_t)l * m + e], Linvt[(int64_t)l * k + j], acc);
        R[t] = acc;
    }
}

// a[i][:] = R^T w_i for test points (k-vectors, row-major ns x k); off-grid points get zeros
template <typename TX, int D>
__global__ void k_lowrank_a(const TX *__restrict__ Xs, int64_t ns, KeyParams kp, const double *__restrict__ R, int k,
                            double *__restrict__ a, int64_t s1, int64_t s2, int *__restrict__ status) {
    const int64_t total = ns * (int64_t)k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k;
        const int l = (int)(t % k);
        int bad = 0;
        // the column l of R as a grid vector is R[node * k + l]: gather with the prediction weights
        int c[3] = {1, 1, 1};
        TX tt[3] = {TX(0), TX(0), TX(0)};
        int st = 0;
#pragma unroll
        for (int q = 0; q < D; ++q) st |= axis_cell<TX>(Xs[(int64_t)q * ns + i], kp, q, c[q], tt[q]);
        if (st) {
            bad |= (st & 2) ? ST_NONFINITE : ST_OUT_OF_GRID;
            a[t] = 0.0;
            if (l == 0) atomicOr(status, bad);
            continue;
        }
        double w[3][4];
#pragma unroll
        for (int q = 0; q < D; ++q) {
            TX wx[4];
            keys_weights<TX>(tt[q], wx);
#pragma unroll
            for (int b = 0; b < 4; ++b) w[q][b] = (double)wx[b];
        }
        double acc = 0.0;
        for (int a0 = 0; a0 < 4; ++a0)
            for (int a1 = 0; a1 < (D > 1 ? 4 : 1); ++a1) {
                double row = 0.0;
                for (int a2 = 0; a2 < (D > 2 ? 4 : 1); ++a2) {
                    int64_t node;
                    double wv;
                    if (D == 1) { node = c[0] - 1 + a0; wv = 1.0; }
                    else if (D == 2) { node = (int64_t)(c[0] - 1 + a0) * s1 + (c[1] - 1 + a1); wv = 1.0; }
                    else { node = (int64_t)(c[0] - 1 + a0) * s1 + (int64_t)(c[1] - 1 + a1) * s2 + (c[2] - 1 + a2); wv = w[2][a2]; }
                    row = fma(wv, R[node * k + l], row);
                }
                acc = fma(w[0][a0] * (D > 1 ? w[1][a1] : 1.0), row, acc);
            }
        a[t] = acc;
    }
}

// cov[i][j] -= a_i . a_j
__global__ void k_lowrank_sub(const double *__restrict__ a, int k, int64_t ns, double *__restrict__ cov) {
    const int64_t total = ns * ns;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / ns, j = t % ns;
        double acc = 0.0;
        for (int l = 0; l < k; ++l) acc = fma(a[i * k + l], a[j * k + l], acc);
        cov[t] -= acc;
    }
}

template <typename TB>
// probe < 0: start at y and build the covariance factor R in st.  probe >= 0: start at the probe
// z_probe (its W^T z and ||z||^2 from the precompute) and return the tridiagonal T (diagonal,
// couplings) for a Lanczos quadrature instead.
static int efla_build(fkski_stats *st, const fkski_kernel *kern, int k, fkski_info *info, cudaStream_t s,
                      int probe = -1, std::vector<double> *tri_dg = nullptr, std::vector<double> *tri_of = nullptr) {
    const int64_t m = st->m;
    const double s2 = kern->noise_var;
    SolveWork *w;
    FK_TRY(work_get(st, &w));
    KgOp *kg64;
    FK_TRY(work_kg(st, w, FKSKI_F64, &kg64));
    FK_TRY(kgop_set(kg64, kern, -1, s));
    const TB *band = (const TB *)st->band;
    const unsigned gb = (unsigned)grid_blocks(m);
    const unsigned gv = (unsigned)std::min<int64_t>(cdiv(m, 256), 152 * 8);
    // device buffers: Qh, Ph (m x (k+1)), wtb, kwb, sh, qn, qprev, G, vectors of scalars
    double *buf = nullptr;
    const size_t nv = (size_t)m;
    const size_t need = nv * (2 * (size_t)(k + 1) + 6) + 4 * (size_t)(k + 1) + 64;
    FK_TRY(pool_alloc((void **)&buf, sizeof(double) * need, s));
    double *Qh = buf, *Ph = Qh + nv * (k + 1), *wtb = Ph + nv * (k + 1), *kwb = wtb + nv, *sh = kwb + nv;
    double *qn = sh + nv, *tmp = qn + nv, *tmp2 = tmp + nv, *lam = tmp2 + nv, *dsc = lam + (k + 1);
    double *sums = dsc + 2 * (k + 1);
    // W^T b = W^T b_in / ||b_in|| (FP64), K W^T b
    const size_t es = st->dtype == FKSKI_F64 ? 8 : 4;
    const void *src = probe < 0 ? st->wty : (const void *)((const char *)st->wtz + (size_t)probe * m * es);
    const double ynorm = std::sqrt(std::max(probe < 0 ? st->yty : st->ztz[probe], 1e-300));
    k_convert<double><<<gv, 256, 0, s>>>(src, st->dtype == FKSKI_F64, wtb, m);
    FK_LAUNCH();
    k_scale_d<<<gv, 256, 0, s>>>(wtb, 1.0 / ynorm, m);
    FK_LAUNCH();
    FK_TRY(kgop_apply(kg64, wtb, kwb, 1, nullptr, 0.0, s));
    FK_CUDA(cudaMemsetAsync(Qh, 0, sizeof(double) * nv * 2 * (k + 1), s));
    FK_CUDA(cudaMemsetAsync(sh, 0, sizeof(double) * nv, s));
    std::vector<double> T((size_t)k * k, 0.0), d(k + 1, 0.0), qw(k + 1, 0.0);
    auto dots = [&](const double *a0, const double *b0, const double *a1, const double *b1, const double *a2,
                    const double *b2, double *out3) -> int {
        k_dots4<double, double><<<gb, CG_T, 0, s>>>(a0, b0, a1, b1, a2, b2, nullptr, nullptr, m, 1, w->part, nullptr);
        k_fin_sums<<<1, 128, 0, s>>>(w->part, gb, 1, 4, sums);
        FK_LAUNCH();
        double h[4];
        FK_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s));
        FK_CUDA(cudaStreamSynchronize(s));
        out3[0] = h[0];
        out3[1] = h[1];
        out3[2] = h[2];
        return FKSKI_OK;
    };
    // q_1 = b: q_hat_1 = 0 (column 0), c_1 = 1
    double c = 1.0, c_prev = 0.0, beta = 0.0;
    d[0] = 1.0;
    qw[0] = 0.0;  // q_hat_1 . W^T b
    int kk = k;
    double *qprev = tmp2;
    FK_CUDA(cudaMemsetAsync(qprev, 0, sizeof(double) * nv, s));
    for (int i = 0; i < k; ++i) {
        double *qi = Qh + nv * i, *pi = Ph + nv * i;
        // q_{i+1} = A q_i - beta_i q_{i-1}  (compressed: s_hat_i + c_i K W^T b - beta_i q_hat_{i-1})
        k_efla_next<<<gv, 256, 0, s>>>(qn, sh, kwb, qprev, c, beta, m);
        FK_LAUNCH();
        const double cn0 = s2 * c - beta * c_prev;
        double t3[3];
        FK_TRY(dots(pi, qn, qn, wtb, qi, wtb, t3));  // P_hat_i.qn, qn.W^T b, q_hat_i.W^T b
        const double alpha = t3[0] + c * cn0 + c * t3[1] + cn0 * t3[2];
        T[(size_t)i * k + i] = alpha;
        if (i == k - 1) break;
        // q_{i+1} -= alpha q_i; then two passes of full reorthogonalisation against q_1..q_i
        k_axpy_d<<<gv, 256, 0, s>>>(qn, qi, -alpha, m);
        FK_LAUNCH();
        double cn = cn0 - alpha * c;
        for (int pass = 0; pass < 2; ++pass) {
            k_gemv_t<<<i + 1, 256, 0, s>>>(Ph, i + 1, m, qn, lam);  // P_hat_j . q_hat_{i+1}
            FK_LAUNCH();
            FK_TRY(dots(qn, wtb, qn, wtb, qn, wtb, t3));             // q_hat_{i+1} . W^T b
            std::vector<double> L(i + 1);
            FK_CUDA(cudaMemcpyAsync(L.data(), lam, sizeof(double) * (i + 1), cudaMemcpyDeviceToHost, s));
            FK_CUDA(cudaStreamSynchronize(s));
            double dl = 0.0;
            for (int j = 0; j <= i; ++j) {
                L[j] += d[j] * cn + d[j] * t3[0] + cn * qw[j];
                dl += d[j] * L[j];
            }
            FK_CUDA(cudaMemcpyAsync(lam, L.data(), sizeof(double) * (i + 1), cudaMemcpyHostToDevice, s));
            k_gemv_sub<<<gv, 256, 0, s>>>(Qh, i + 1, m, lam, qn);
            FK_LAUNCH();
            cn -= dl;
        }
        // B(q_hat_{i+1}): P_hat = W^T W q_hat, s_hat = K P_hat + sigma^2 q_hat
        double *pn = Ph + nv * (i + 1);
        FK_TRY((launch_spmv<TB, double>(band, st->grid, qn, pn, m, 1, nullptr, 1, nullptr, nullptr, gb, s)));
        FK_TRY(kgop_apply(kg64, pn, sh, 1, qn, s2, s));
        FK_TRY(dots(pn, qn, qn, wtb, qn, qn, t3));  // P.q, q.W^T b, q.q
        const double b2 = t3[0] + cn * cn + 2.0 * cn * t3[1];
        const double scale_ref = std::fabs(alpha) + std::fabs(beta) + 1e-300;
        if (!(b2 > 0.0) || std::sqrt(b2) <= 1e-10 * scale_ref) {  // invariant Krylov space
            kk = i + 1;
            break;
        }
        const double bn = std::sqrt(b2);
        T[(size_t)i * k + i + 1] = T[(size_t)(i + 1) * k + i] = bn;
        FK_CUDA(cudaMemcpyAsync(qprev, qi, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
        k_scale_d<<<gv, 256, 0, s>>>(qn, 1.0 / bn, m);
        k_scale_d<<<gv, 256, 0, s>>>(pn, 1.0 / bn, m);
        k_scale_d<<<gv, 256, 0, s>>>(sh, 1.0 / bn, m);
        FK_LAUNCH();
        FK_CUDA(cudaMemcpyAsync(Qh + nv * (i + 1), qn, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
        c_prev = c;
        c = cn / bn;
        beta = bn;
        d[i + 1] = c;
        qw[i + 1] = t3[1] / bn;
    }
    if (probe >= 0) {
        tri_dg->assign(kk, 0.0);
        tri_of->assign(kk, 0.0);
        for (int i = 0; i < kk; ++i) {
            (*tri_dg)[i] = T[(size_t)i * k + i];
            if (i + 1 < kk) (*tri_of)[i] = T[(size_t)i * k + i + 1];
        }
        cudaFreeAsync(buf, s);
        FK_CUDA(cudaStreamSynchronize(s));
        if (info) info->iters = std::max(info->iters, kk);
        return FKSKI_OK;
    }
    // T = L L^T (host), Linv^T
    std::vector<double> Lm((size_t)kk * kk, 0.0), Li((size_t)kk * kk, 0.0);
    for (int j = 0; j < kk; ++j) {
        double sum = T[(size_t)j * k + j];
        for (int l = 0; l < j; ++l) sum -= Lm[(size_t)j * kk + l] * Lm[(size_t)j * kk + l];
        if (!(sum > 0.0)) {
            cudaFreeAsync(buf, s);
            return FKSKI_E_BREAKDOWN;
        }
        Lm[(size_t)j * kk + j] = std::sqrt(sum);
        for (int r = j + 1; r < kk; ++r) {
            double v = T[(size_t)r * k + j];
            for (int l = 0; l < j; ++l) v -= Lm[(size_t)r * kk + l] * Lm[(size_t)j * kk + l];
            Lm[(size_t)r * kk + j] = v / Lm[(size_t)j * kk + j];
        }
    }
    // Li = L^{-1} (lower); Linv^T[l][j] = Li[j][l]
    for (int j = 0; j < kk; ++j) {
        Li[(size_t)j * kk + j] = 1.0 / Lm[(size_t)j * kk + j];
        for (int r = j + 1; r < kk; ++r) {
            double v = 0.0;
            for (int l = j; l < r; ++l) v += Lm[(size_t)r * kk + l] * Li[(size_t)l * kk + j];
            Li[(size_t)r * kk + j] = -v / Lm[(size_t)r * kk + r];
        }
    }
    std::vector<double> Lt((size_t)kk * kk, 0.0);
    for (int l = 0; l < kk; ++l)
        for (int j = 0; j < kk; ++j) Lt[(size_t)l * kk + j] = Li[(size_t)j * kk + l];
    // G = K (P_hat + W^T b d^T), column-major m x kk (overwrites Q_hat's storage)
    double *G = Qh;
    FK_CUDA(cudaMemcpyAsync(G, Ph, sizeof(double) * nv * kk, cudaMemcpyDeviceToDevice, s));
    for (int j = 0; j < kk; ++j) {
        k_axpy_d<<<gv, 256, 0, s>>>(G + nv * j, wtb, d[j], m);
        FK_LAUNCH();
    }
    FK_TRY(kgop_apply(kg64, G, Ph, kk, nullptr, 0.0, s));  // Ph <- K G
    double *dLt = nullptr;
    FK_TRY(pool_alloc((void **)&dLt, sizeof(double) * kk * kk, s));
    FK_CUDA(cudaMemcpyAsync(dLt, Lt.data(), sizeof(double) * kk * kk, cudaMemcpyHostToDevice, s));
    if (st->lowrank) cudaFree(st->lowrank);
    st->lowrank = nullptr;
    FK_TRY(dev_alloc((void **)&st->lowrank, sizeof(double) * nv * kk));
    const unsigned gr = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv((int64_t)nv * kk, 256), 152 * 16));
    k_lowrank_R<<<gr, 256, 0, s>>>(Ph, dLt, kk, m, st->lowrank);
    FK_LAUNCH();
    cudaFreeAsync(dLt, s);
    cudaFreeAsync(buf, s);
    FK_CUDA(cudaStreamSynchronize(s));
    st->lowrank_k = kk;
    st->lowrank_kreq = k;
    st->lowrank_kern = *kern;
    if (info) {
        info->iters = kk;
        info->status = FKSKI_OK;
    }
    return FKSKI_OK;
}

// Lanczos tridiagonal of A started at probe z_p (EFLA, k steps, full reorthogonalisation).
int efla_probe_tridiag(fkski_stats *st, const fkski_kernel *kern, int k, int probe, std::vector<double> &dg,
                       std::vector<double> &of, fkski_info *info, cudaStream_t s) {
    if (!st || !kern || k < 1 || probe < 0 || probe >= st->nprobes) return FKSKI_E_INVALID_ARG;
    return st->dtype == FKSKI_F32 ? efla_build<float>(st, kern, k, info, s, probe, &dg, &of)
                                  : efla_build<double>(st, kern, k, info, s, probe, &dg, &of);
}

static bool same_kernel(const fkski_kernel &a, const fkski_kernel &b, int d) {
    if (a.type != b.type || a.outputscale != b.outputscale || a.noise_var != b.noise_var) return false;
    for (int k = 0; k < d; ++k)
        if (a.lengthscale[k] != b.lengthscale[k]) return false;
    return true;
}

template <typename TX>
static int lowrank_eval(fkski_stats *st, const fkski_kernel *kern, const TX *Xs, int64_t ns, double *cov, cudaStream_t s) {
    const int64_t m = st->m;
    const int d = st->d, k = st->lowrank_k;
    const KeyParams kp = make_key_params(st->grid);
    const int64_t M1 = st->grid.M[1], M2 = st->grid.M[2];
    const int64_t s1 = d == 2 ? M1 : M1 * M2, s2 = M2;
    SolveWork *w;
    FK_TRY(work_get(st, &w));
    KgOp *kg64;
    FK_TRY(work_kg(st, w, FKSKI_F64, &kg64));
    FK_TRY(kgop_set(kg64, kern, -1, s));
    double *e = nullptr, *kw = nullptr, *a = nullptr;
    int *dstatus = nullptr;
    const size_t nR = (size_t)COV_R * m;
    FK_TRY(pool_alloc((void **)&e, sizeof(double) * nR, s));
    FK_TRY(pool_alloc((void **)&kw, sizeof(double) * nR, s));
    FK_TRY(pool_alloc((void **)&a, sizeof(double) * (size_t)ns * k, s));
    FK_TRY(pool_alloc((void **)&dstatus, sizeof(int), s));
    FK_CUDA(cudaMemsetAsync(dstatus, 0, sizeof(int), s));
    // prior w_i^T K w_j, a block of test points per K_G product
    for (int64_t j0 = 0; j0 < ns; j0 += COV_R) {
        const int R = (int)std::min<int64_t>(COV_R, ns - j0);
        FK_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * R * m, s));
        if (d == 1) k_scatter_w<TX, 1><<<(R + 63) / 64, 64, 0, s>>>(Xs, ns, j0, R, kp, e, m, s1, s2, dstatus);
        else if (d == 2) k_scatter_w<TX, 2><<<(R + 63) / 64, 64, 0, s>>>(Xs, ns, j0, R, kp, e, m, s1, s2, dstatus);
        else k_scatter_w<TX, 3><<<(R + 63) / 64, 64, 0, s>>>(Xs, ns, j0, R, kp, e, m, s1, s2, dstatus);
        FK_LAUNCH();
        FK_TRY(kgop_apply(kg64, e, kw, R, nullptr, 0.0, s));
        const unsigned gg = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(ns * R, 256), 152 * 16));
        if (d == 1) k_cov_gather<TX, 1><<<gg, 256, 0, s>>>(Xs, ns, kp, kw, R, m, j0, cov, s1, s2);
        else if (d == 2) k_cov_gather<TX, 2><<<gg, 256, 0, s>>>(Xs, ns, kp, kw, R, m, j0, cov, s1, s2);
        else k_cov_gather<TX, 3><<<gg, 256, 0, s>>>(Xs, ns, kp, kw, R, m, j0, cov, s1, s2);
        FK_LAUNCH();
    }
    const unsigned ga = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(ns * k, 256), 152 * 16));
    if (d == 1) k_lowrank_a<TX, 1><<<ga, 256, 0, s>>>(Xs, ns, kp, st->lowrank, k, a, s1, s2, dstatus);
    else if (d == 2) k_lowrank_a<TX, 2><<<ga, 256, 0, s>>>(Xs, ns, kp, st->lowrank, k, a, s1, s2, dstatus);
    else k_lowrank_a<TX, 3><<<ga, 256, 0, s>>>(Xs, ns, kp, st->lowrank, k, a, s1, s2, dstatus);
    FK_LAUNCH();
    const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(ns * ns, 256), 152 * 16));
    k_lowrank_sub<<<gs, 256, 0, s>>>(a, k, ns, cov);
    FK_LAUNCH();
    int hst = 0;
    FK_CUDA(cudaMemcpyAsync(&hst, dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(e, s);
    cudaFreeAsync(kw, s);
    cudaFreeAsync(a, s);
    cudaFreeAsync(dstatus, s);
    FK_CUDA(cudaStreamSynchronize(s));
    return status_from_bits(hst);
}

int posterior_cov_lowrank_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, int k, const void *Xs,
                               int xdtype, int64_t ns, double *cov, fkski_info *info, cudaStream_t s) {
    (void)opts;
    if (!st || !kern || k < 1 || ns < 0 || (ns > 0 && (!Xs || !cov))) return FKSKI_E_INVALID_ARG;
    if (!(kern->noise_var > 0.0) || !std::isfinite(kern->noise_var)) return FKSKI_E_INVALID_ARG;
    if (xdtype != FKSKI_F32 && xdtype != FKSKI_F64) return FKSKI_E_INVALID_ARG;
    if (info) memset(info, 0, sizeof(*info));
    if (!st->lowrank || st->lowrank_kreq != k || !same_kernel(st->lowrank_kern, *kern, st->d)) {
        const int rc = st->dtype == FKSKI_F32 ? efla_build<float>(st, kern, k, info, s) : efla_build<double>(st, kern, k, info, s);
        if (rc != FKSKI_OK) return rc;
    } else if (info) {
        info->iters = st->lowrank_k;
    }
    if (ns == 0) return FKSKI_OK;
    return xdtype == FKSKI_F32 ? lowrank_eval<float>(st, kern, (const float *)Xs, ns, cov, s)
                               : lowrank_eval<double>(st, kern, (const double *)Xs, ns, cov, s);
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
