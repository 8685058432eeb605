// Plain SKI (Def. 1) posterior mean by n-space CG (Alg. 1) on A = W K_G W^T + sigma^2 I: the
// O(n + m log m)-per-iteration baseline the paper's factorized methods are compared with
// (Sec. 5, Fig. 2 and Table 1).  Each iteration applies W^T (a per-cell reduction over the points
// in cell order, then each grid node sums the 4^d cells around it), K_G (the same FFT passes as
// the factorized solver) and W (a 4^d gather per point), plus n-space vector updates.
//
// n-space vectors are kept in cell order (the order of the points kept by the precompute with
// opts.keep_points), so every pass streams the points and each cell's reduction reads a
// contiguous segment; the permutation is never applied per iteration.  Inner products: in the
// vector type within a warp, FP64 across warps and blocks in a fixed order.  Scalars live on the
// device; iterations run as captured CUDA-graph chunks like the factorized solver.
//
// Precision follows the factorized solver's modes: vectors of type T (FP32, FP64, or double-float
// for MIXED) over points stored in TP.  W's entry for point i and stencil node a is the product
// w_{a_1}(t_i1) ... w_{a_d}(t_id) rounded once in TP, and W and W^T both use exactly that value
// (W^T is the exact transpose of the W applied); sums over points or nodes accumulate in T (the
// lazily normalised double-float sum for MIXED).
#include "fkski_internal.cuh"

#include <algorithm>
#include <vector>

namespace fk {

constexpr int SKI_T = 256;

template <int D>
struct NA {
    static constexpr int v = D == 1 ? 4 : (D == 2 ? 16 : 64);
};

// Accumulators for sums of (TP weight) x (T value): plain FMA for FP32 / FP64 vectors, the
// lazily normalised double-float sum for double-float vectors.
template <typename T>
struct SkiAcc {
    T v;
    __device__ __forceinline__ void zero() { v = T(0); }
    template <typename TP>
    __device__ __forceinline__ void add(TP w, T x) { v = fma((T)w, x, v); }
    __device__ __forceinline__ T value() const { return v; }
};
template <>
struct SkiAcc<dfl> {
    dacc a;
    __device__ __forceinline__ void zero() { dacc_zero(a); }
    __device__ __forceinline__ void add(float w, dfl x) { dacc_add_fx(a, w, x); }
    __device__ __forceinline__ dfl value() const { return dacc_value(a); }
};

// Sum over a warp (fixed butterfly tree).
__device__ __forceinline__ float warp_sum_t(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}
__device__ __forceinline__ double warp_sum_t(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}
__device__ __forceinline__ dfl warp_sum_t(dfl x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        x = x + dfl(__shfl_xor_sync(0xFFFFFFFFu, x.hi, o), __shfl_xor_sync(0xFFFFFFFFu, x.lo, o));
    return x;
}

// W's entry for stencil node a (digits a_k = bits 2k..2k+1 from the last axis) of a point with
// weights w: the product over axes, rounded once in TP, axis 0 first.
template <typename TP, int D>
__device__ __forceinline__ TP w_entry(const TP (&w)[3][4], int a) {
    int dg[3] = {0, 0, 0};
    int rem = a;
#pragma unroll
    for (int q = D - 1; q >= 0; --q) {
        dg[q] = rem & 3;
        rem >>= 2;
    }
    TP e = w[0][dg[0]];
#pragma unroll
    for (int q = 1; q < D; ++q) e *= w[q][dg[q]];
    return e;
}

// cell key -> the first stencil node of the cell (cell index c - 1 on each axis = key digit)
struct SkiGeom {
    int d;
    int64_t ncell[3];  // cells per axis (M_k - 3)
    int64_t M[3];
};

__device__ __forceinline__ void key_digits(uint32_t key, const SkiGeom &g, int64_t c[3]) {
    int64_t r = key;
    for (int k = g.d - 1; k >= 0; --k) {
        c[k] = r % g.ncell[k];
        r /= g.ncell[k];
    }
}

// Per cell: Yc[a] = sum_{points i in the cell} v_i prod_k w_{a_k}(t_ik), a in [0,4)^d.
// One warp per cell, lanes stride over the points; fixed shuffle tree (deterministic).
template <typename TP, typename T, int D>
__global__ void __launch_bounds__(SKI_T) k_ski_cells(const Rec4<TP> *__restrict__ pts, const uint32_t *__restrict__ off,
                                                     int64_t ncells, const T *__restrict__ v, T *__restrict__ yc,
                                                     const int *__restrict__ gate) {
    if (gate && *gate) return;
    constexpr int NA_ = NA<D>::v;
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = wg; c < ncells; c += nw) {
        const uint32_t beg = off[c], end = off[c + 1];
        SkiAcc<T> acc[NA_];
#pragma unroll
        for (int a = 0; a < NA_; ++a) acc[a].zero();
        for (uint32_t k = beg + lane; k < end; k += 32) {
            const Rec4<TP> r = pts[k];
            const T vk = v[k];
            TP w[3][4];
#pragma unroll
            for (int q = 0; q < D; ++q) keys_weights<TP>(r.t[q], w[q]);
#pragma unroll
            for (int a = 0; a < NA_; ++a) acc[a].add(w_entry<TP, D>(w, a), vk);
        }
#pragma unroll
        for (int a = 0; a < NA_; ++a) {
            const T x = warp_sum_t(acc[a].value());
            if (lane == 0) yc[c * NA_ + a] = x;
        }
    }
}

// u[j] = sum_a Yc[j - a][a]: grid node j collects the 4^d cells whose stencil holds it.
template <typename T, int D>
__global__ void k_ski_nodes(const T *__restrict__ yc, SkiGeom g, int64_t m, T *__restrict__ u, const int *__restrict__ gate) {
    if (gate && *gate) return;
    constexpr int NA_ = NA<D>::v;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t jj[3] = {0, 0, 0};
        int64_t r = j;
        for (int k = D - 1; k >= 0; --k) {
            jj[k] = r % g.M[k];
            r /= g.M[k];
        }
        T acc = T(0);
#pragma unroll
        for (int a = 0; a < NA_; ++a) {
            int rem = a;
            int64_t key = 0;
            bool ok = true;
#pragma unroll
            for (int k = D - 1; k >= 0; --k) {
                const int ak = rem & 3;
                rem >>= 2;
                const int64_t c = jj[k] - ak;
                ok = ok && c >= 0 && c < g.ncell[k];
                key = key + c * (k == D - 1 ? 1 : (k == D - 2 ? g.ncell[D - 1] : g.ncell[D - 1] * g.ncell[D - 2]));
            }
            if (ok) acc += yc[key * NA_ + a];
        }
        u[j] = acc;
    }
}

// ap_k = (W ku)_k + sigma^2 p_k (per point, cell order), partial p.ap per block.
template <typename TP, typename T, int D>
__global__ void __launch_bounds__(SKI_T) k_ski_ap(const Rec4<TP> *__restrict__ pts, const uint32_t *__restrict__ pkeys,
                                                  int64_t n, SkiGeom g, const T *__restrict__ ku, const T *__restrict__ p,
                                                  T *__restrict__ ap, const double *__restrict__ sig2,
                                                  double *__restrict__ part, const int *__restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[SKI_T / 32];
    const T s2 = (T)(*sig2);
    T dq = T(0);
    int64_t s1 = 1, s2s = 1;
    if (D == 2) s1 = g.M[1];
    if (D == 3) { s1 = g.M[1] * g.M[2]; s2s = g.M[2]; }
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const Rec4<TP> r = pts[k];
        int64_t c[3] = {0, 0, 0};
        key_digits(pkeys[k], g, c);
        TP w[3][4];
#pragma unroll
        for (int q = 0; q < D; ++q) keys_weights<TP>(r.t[q], w[q]);
        SkiAcc<T> acc;
        acc.zero();
#pragma unroll
        for (int a = 0; a < NA<D>::v; ++a) {
            const int a0 = D == 1 ? a : (D == 2 ? (a >> 2) : (a >> 4));
            const int a1 = D == 2 ? (a & 3) : ((a >> 2) & 3), a2 = a & 3;
            const int64_t node = D == 1 ? c[0] + a0
                               : (D == 2 ? (c[0] + a0) * s1 + c[1] + a1 : (c[0] + a0) * s1 + (c[1] + a1) * s2s + c[2] + a2);
            acc.add(w_entry<TP, D>(w, a), ku[node]);
        }
        const T pk = p[k];
        const T v = fma(s2, pk, acc.value());
        ap[k] = v;
        dq = fma(pk, v, dq);
    }
    double t = (double)dq;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w2 = 0; w2 < SKI_T / 32; ++w2) s += sh[w2];
        part[blockIdx.x] = s;
    }
}

// Scalars: sc[0] gamma = r.r, sc[1] alpha, sc[2] beta, sc[3] eps, sc[4] last residual;
// flags[0] done, flags[1] iterations, flags[2] breakdown, flags[3] maxiter.
__global__ void k_ski_alpha(const double *__restrict__ part, int nparts, double *__restrict__ sc, int *__restrict__ flags) {
    if (flags[0]) return;
    __shared__ double sh[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        if (!(t > 0.0) || !isfinite(t)) {
            flags[0] = 1;
            flags[2] = 1;
        } else {
            sc[1] = sc[0] / t;
        }
    }
}

// x += alpha p, r -= alpha ap; partial r.r
template <typename T>
__global__ void __launch_bounds__(SKI_T) k_ski_xr(int64_t n, T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                                                  const T *__restrict__ ap, const double *__restrict__ sc,
                                                  double *__restrict__ part, const int *__restrict__ flags) {
    if (flags[0]) return;
    __shared__ double sh[SKI_T / 32];
    const T a = (T)sc[1];
    T dq = T(0);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        x[k] = fma(a, p[k], x[k]);
        const T rk = fma(-a, ap[k], r[k]);
        r[k] = rk;
        dq = fma(rk, rk, dq);
    }
    double t = (double)dq;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w2 = 0; w2 < SKI_T / 32; ++w2) s += sh[w2];
        part[blockIdx.x] = s;
    }
}

__global__ void k_ski_beta(const double *__restrict__ part, int nparts, double *__restrict__ sc, int *__restrict__ flags) {
    if (flags[0]) return;
    __shared__ double sh[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double g = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) g += sh[w];
        flags[1] += 1;
        sc[4] = g;
        if (!isfinite(g)) {
            flags[0] = 1;
            flags[2] = 1;
        } else if (g <= sc[3] || flags[1] >= flags[3]) {
            flags[0] = 1;
        } else {
            sc[2] = g / sc[0];
            sc[0] = g;
        }
    }
}

template <typename T>
__global__ void k_ski_p(int64_t n, T *__restrict__ p, const T *__restrict__ r, const double *__restrict__ sc,
                        const int *__restrict__ flags) {
    if (flags[0]) return;
    const T b = (T)sc[2];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        p[k] = fma(b, p[k], r[k]);
}

template <typename TP, typename T>
__global__ void k_ski_init(int64_t n, const Rec4<TP> *__restrict__ pts, T *__restrict__ x, T *__restrict__ r,
                           T *__restrict__ p) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const T y = T(pts[k].y);
        x[k] = T(0);
        r[k] = y;
        p[k] = y;
    }
}

template <typename T>
__global__ void k_ski_out(const T *__restrict__ in, OutT<T> *__restrict__ out, int64_t m) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (OutT<T>)(double)in[e];
}

template <typename TP, typename T, int D>
static void launch_wt(const Rec4<TP> *pts, const uint32_t *off, int64_t ncells, const SkiGeom &g, int64_t m, const T *v,
                      T *yc, T *u, const int *gate, cudaStream_t s) {
    const unsigned gc = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(ncells * 32, SKI_T), 152 * 16));
    k_ski_cells<TP, T, D><<<gc, SKI_T, 0, s>>>(pts, off, ncells, v, yc, gate);
    const unsigned gn = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(m, 256), 152 * 8));
    k_ski_nodes<T, D><<<gn, 256, 0, s>>>(yc, g, m, u, gate);
}

template <typename TP, typename T, int D>
static int ski_typed(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *o, OutT<T> *a_out, OutT<T> *v_out,
                     fkski_info *info, cudaStream_t s) {
    const int64_t n = st->n, m = st->m, ncells = st->ncells;
    constexpr int NA_ = NA<D>::v;
    SkiGeom g;
    memset(&g, 0, sizeof(g));
    g.d = D;
    for (int k = 0; k < D; ++k) {
        g.ncell[k] = st->grid.M[k] - 3;
        g.M[k] = st->grid.M[k];
    }
    const Rec4<TP> *pts = (const Rec4<TP> *)st->pts;
    // operator and buffers
    KgOp *kg = nullptr;
    FK_TRY(kgop_create(&st->grid, dtype_of<T>(), &kg));
    struct Guard {
        KgOp *kg;
        std::vector<void *> bufs;
        cudaStream_t s;
        ~Guard() {
            cudaStreamSynchronize(s);
            for (void *b : bufs) cudaFreeAsync(b, s);
            cudaStreamSynchronize(s);
            kgop_destroy(kg);
        }
    } guard{kg, {}, s};
    auto get = [&](void **p, size_t bytes) -> int {
        FK_TRY(pool_alloc(p, bytes, s));
        guard.bufs.push_back(*p);
        return FKSKI_OK;
    };
    T *x, *r, *p, *ap, *u, *ku, *yc, *aT, *vT;
    double *part, *sc, *sig2;
    int *flags;
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, SKI_T), 152 * 8));
    FK_TRY(get((void **)&x, sizeof(T) * n));
    FK_TRY(get((void **)&r, sizeof(T) * n));
    FK_TRY(get((void **)&p, sizeof(T) * n));
    FK_TRY(get((void **)&ap, sizeof(T) * n));
    FK_TRY(get((void **)&u, sizeof(T) * m));
    FK_TRY(get((void **)&ku, sizeof(T) * m));
    FK_TRY(get((void **)&yc, sizeof(T) * ncells * NA_));
    FK_TRY(get((void **)&aT, sizeof(T) * m));
    FK_TRY(get((void **)&vT, sizeof(T) * m));
    FK_TRY(get((void **)&part, sizeof(double) * gb));
    FK_TRY(get((void **)&sc, sizeof(double) * 8));
    FK_TRY(get((void **)&sig2, sizeof(double)));
    FK_TRY(get((void **)&flags, sizeof(int) * 4));
    FK_TRY(kgop_set(kg, kern, -1, s));
    FK_TRY(kgop_reserve(kg, 1));
    FK_TRY(kgop_tune(kg, 1, s));
    // x0 = 0, r0 = p0 = y (cell order); gamma0 = y^T y, eps = rtol^2 y^T y
    const double hs[8] = {st->yty, 0.0, 0.0, o->rtol * o->rtol * st->yty, st->yty, 0.0, 0.0, 0.0};
    const int hf[4] = {0, 0, 0, o->maxiter};
    const double s2v = kern->noise_var;
    FK_CUDA(cudaMemcpyAsync(sc, hs, sizeof(hs), cudaMemcpyHostToDevice, s));
    FK_CUDA(cudaMemcpyAsync(flags, hf, sizeof(hf), cudaMemcpyHostToDevice, s));
    FK_CUDA(cudaMemcpyAsync(sig2, &s2v, sizeof(double), cudaMemcpyHostToDevice, s));
    k_ski_init<TP, T><<<gb, SKI_T, 0, s>>>(n, pts, x, r, p);
    FK_LAUNCH();
    // capture a chunk of iterations on an internal stream
    cudaStream_t cs;
    FK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t ev;
    FK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    const int check = std::max(1, o->check_every);
    const long long before = fkski_kernel_launches();
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = FKSKI_OK;
    kgop_set_gate(kg, flags);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    for (int it = 0; it < check && e == cudaSuccess && rc == FKSKI_OK; ++it) {
        launch_wt<TP, T, D>(pts, st->offsets, ncells, g, m, p, yc, u, flags, cs);
        rc = kgop_apply(kg, u, ku, 1, nullptr, 0.0, cs);
        if (rc) break;
        k_ski_ap<TP, T, D><<<gb, SKI_T, 0, cs>>>(pts, st->pkeys, n, g, ku, p, ap, sig2, part, flags);
        k_ski_alpha<<<1, 256, 0, cs>>>(part, (int)gb, sc, flags);
        k_ski_xr<T><<<gb, SKI_T, 0, cs>>>(n, x, r, p, ap, sc, part, flags);
        k_ski_beta<<<1, 256, 0, cs>>>(part, (int)gb, sc, flags);
        k_ski_p<T><<<gb, SKI_T, 0, cs>>>(n, p, r, sc, flags);
    }
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    kgop_set_gate(kg, nullptr);
    if (e == cudaSuccess) e = ec;
    size_t nn = 0;
    if (e == cudaSuccess && rc == FKSKI_OK) e = cudaGraphGetNodes(graph, nullptr, &nn);
    count_launches(before - fkski_kernel_launches());
    if (e == cudaSuccess && rc == FKSKI_OK) e = cudaGraphInstantiate(&exec, graph, 0);
    int *hflags = nullptr;
    if (e == cudaSuccess && rc == FKSKI_OK) e = cudaMallocHost((void **)&hflags, sizeof(int) * 4);
    if (e == cudaSuccess && rc == FKSKI_OK) {
        e = cudaEventRecord(ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
        for (int launched = 0; e == cudaSuccess && launched <= o->maxiter + check; launched += check) {
            e = cudaGraphLaunch(exec, cs);
            count_launches((long long)nn);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
            if (e == cudaSuccess && hflags[0]) break;
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
    cudaEventDestroy(ev);
    if (rc == FKSKI_OK && e != cudaSuccess) rc = note_cuda_error(e, __FILE__, __LINE__);
    int hf2[4] = {0, 0, 0, 0};
    double hs2[8];
    if (rc == FKSKI_OK) {
        // a = W^T z, v = K_G a (in T, then to the output type)
        launch_wt<TP, T, D>(pts, st->offsets, ncells, g, m, x, yc, aT, nullptr, s);
        FK_LAUNCH();
        rc = kgop_apply(kg, aT, vT, 1, nullptr, 0.0, s);
        if (rc == FKSKI_OK) {
            const unsigned gv = (unsigned)std::min<int64_t>(cdiv(m, 256), 152 * 8);
            k_ski_out<T><<<gv, 256, 0, s>>>(aT, a_out, m);
            k_ski_out<T><<<gv, 256, 0, s>>>(vT, v_out, m);
            FK_LAUNCH();
        }
    }
    if (rc == FKSKI_OK) {
        FK_CUDA(cudaMemcpyAsync(hf2, flags, sizeof(hf2), cudaMemcpyDeviceToHost, s));
        FK_CUDA(cudaMemcpyAsync(hs2, sc, sizeof(hs2), cudaMemcpyDeviceToHost, s));
        FK_CUDA(cudaStreamSynchronize(s));
    }
    if (hflags) cudaFreeHost(hflags);
    if (rc != FKSKI_OK) return rc;
    if (info) {
        info->iters = hf2[1];
        info->iters_rhs[0] = hf2[1];
        info->rel_residual = std::sqrt(std::max(hs2[4], 0.0) / std::max(st->yty, 1e-300));
        info->status = hf2[2] ? FKSKI_E_BREAKDOWN : (hs2[4] > hs2[3] ? FKSKI_E_NOT_CONVERGED : FKSKI_OK);
    }
    if (hf2[2]) return FKSKI_E_BREAKDOWN;
    return hs2[4] > hs2[3] ? FKSKI_E_NOT_CONVERGED : FKSKI_OK;
}

int ski_solve_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, void *a_out, void *v_out,
                   fkski_info *info, cudaStream_t s) {
    if (!st || !kern || !a_out || !v_out) return FKSKI_E_INVALID_ARG;
    if (!st->pts || !st->pkeys || !st->offsets) return FKSKI_E_UNSUPPORTED;  // precompute with keep_points
    fkski_opts o;
    if (opts) o = *opts; else fkski_default_opts(&o);
    if (!(kern->noise_var > 0.0) || !std::isfinite(kern->noise_var)) return FKSKI_E_INVALID_ARG;
    if (o.maxiter < 1 || !(o.rtol >= 0.0)) return FKSKI_E_INVALID_ARG;
    if (info) memset(info, 0, sizeof(*info));
    if (o.precision != FKSKI_MIXED && o.precision != FKSKI_DOUBLE && o.precision != FKSKI_FP32)
        return FKSKI_E_INVALID_ARG;
    // FP32 points: vectors per the precision mode (outputs FP32 except for DOUBLE); FP64 points: FP64
    if (st->dtype == FKSKI_F32) {
        if (o.precision == FKSKI_DOUBLE) {
            double *a = (double *)a_out, *v = (double *)v_out;
            return st->d == 1 ? ski_typed<float, double, 1>(st, kern, &o, a, v, info, s)
                 : st->d == 2 ? ski_typed<float, double, 2>(st, kern, &o, a, v, info, s)
                              : ski_typed<float, double, 3>(st, kern, &o, a, v, info, s);
        }
        float *a = (float *)a_out, *v = (float *)v_out;
        if (o.precision == FKSKI_FP32)
            return st->d == 1 ? ski_typed<float, float, 1>(st, kern, &o, a, v, info, s)
                 : st->d == 2 ? ski_typed<float, float, 2>(st, kern, &o, a, v, info, s)
                              : ski_typed<float, float, 3>(st, kern, &o, a, v, info, s);
        return st->d == 1 ? ski_typed<float, dfl, 1>(st, kern, &o, a, v, info, s)
             : st->d == 2 ? ski_typed<float, dfl, 2>(st, kern, &o, a, v, info, s)
                          : ski_typed<float, dfl, 3>(st, kern, &o, a, v, info, s);
    }
    double *a = (double *)a_out, *v = (double *)v_out;
    return st->d == 1 ? ski_typed<double, double, 1>(st, kern, &o, a, v, info, s)
         : st->d == 2 ? ski_typed<double, double, 2>(st, kern, &o, a, v, info, s)
                      : ski_typed<double, double, 3>(st, kern, &o, a, v, info, s);
}

}  // namespace fk
