// Internal declarations shared by the fkski CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <vector>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "../../include/fkski.h"
#include "dfloat.cuh"

namespace fk {
// Records the failing CUDA call (thread-local) for fkski_last_error_detail(); returns the status.
int note_cuda_error(cudaError_t e, const char *file, int line);
// Stream-ordered temporary from the library's per-device caching pool (free with cudaFreeAsync).
int pool_alloc(void **p, size_t bytes, cudaStream_t s);
// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the current device, never
// lowering it: kernel nodes captured in a CUDA graph keep their sizes, and a later smaller limit
// would make their launches fail.
int raise_smem_limit(const void *func, size_t bytes);
}  // namespace fk

#define FK_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return fk::note_cuda_error(_e, __FILE__, __LINE__); \
    } while (0)

#define FK_TRY(call)                 \
    do {                             \
        int _s = (call);             \
        if (_s != FKSKI_OK) return _s; \
    } while (0)

namespace fk {
// Process-wide count of kernel launches made by this library (graph launches add the number of
// kernel nodes they replay).  Read through fkski_kernel_launches().
void count_launches(long long k);
}  // namespace fk

#define FK_LAUNCH()                    \
    do {                               \
        fk::count_launches(1);         \
        FK_CUDA(cudaGetLastError());   \
    } while (0)

namespace fk {

constexpr int kMaxProbes = 64;

// Element-type code of double-float vectors (dfloat.cuh) next to FKSKI_F32 / FKSKI_F64.
constexpr int FK_DF = FKSKI_F32X2;
template <typename T>
constexpr int dtype_of() {
    return sizeof(T) == 4 ? FKSKI_F32 : (std::is_same<T, dfl>::value ? FK_DF : FKSKI_F64);
}
// Element type of the band matrix a solve in vector type T reads: FP32 for double-float vectors.
template <typename T>
struct BandOf { using type = T; };
template <>
struct BandOf<dfl> { using type = float; };
template <typename T>
using BandT = typename BandOf<T>::type;
// Element type of a solve's output vectors (posterior mean on the grid): FP32 for double-float.
template <typename T>
struct OutOf { using type = T; };
template <>
struct OutOf<dfl> { using type = float; };
template <typename T>
using OutT = typename OutOf<T>::type;
constexpr int kMaxD = 3;

inline int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Device status bits written by kernels (never a trap).
enum : int {
    ST_OUT_OF_GRID = 1,
    ST_NONFINITE = 2,
    ST_BREAKDOWN = 4,
    ST_TIMEOUT = 8,
};

inline int status_from_bits(int bits) {
    if (bits & ST_NONFINITE) return FKSKI_E_NONFINITE;
    if (bits & ST_OUT_OF_GRID) return FKSKI_E_OUT_OF_GRID;
    if (bits & ST_BREAKDOWN) return FKSKI_E_BREAKDOWN;
    if (bits & ST_TIMEOUT) return FKSKI_E_TIMEOUT;
    return FKSKI_OK;
}

// Per-axis constants for the cell index of an FP32 coordinate: lo and 1/h split into float
// pairs on the host, exactly as the key's definition prescribes.
struct AxisKeyF {
    float L1, L2, I1, I2, top;
    int M;
};
struct AxisKeyD {
    double lo, ih;
    int M;
};
struct KeyParams {
    int d;
    AxisKeyF f[3];
    AxisKeyD g[3];
    int64_t cstride[3];  // cell strides (C order over M_k - 3 cells per axis)
    int64_t ncell[3];
};

KeyParams make_key_params(const fkski_grid &g);

// Solver-side workspace kept inside a stats object (see solve.cu).
struct SolveWork;

}  // namespace fk

// The opaque stats object of the C ABI.
struct fkski_stats {
    fkski_grid grid;
    int d;
    int dtype;           // FKSKI_F32 / FKSKI_F64 of the points (and of band/wty/wtz as computed)
    int64_t n, m, ncells;
    int nprobes;
    uint64_t probe_seed;
    double yty;
    double ztz[fk::kMaxProbes];
    int device;
    // sufficient statistics, in `dtype`; from the library's memory pool (returned to it by
    // fkski_destroy, so that repeated precomputes map no new memory)
    void *band;     // 7^d x m
    void *wty;      // m
    void *wtz;      // nprobes x m
    // lazily converted copies in the other precision (for MIXED/DOUBLE solves)
    void *band_alt;
    void *wty_alt;
    void *wtz_alt;
    // W^T y and W^T z as double-float vectors (the MIXED solves), made on first use
    void *wty_df;
    void *wtz_df;
    // optional sort export
    uint32_t *keys;
    uint32_t *perm;
    uint32_t *offsets;  // ncells + 1
    // points in cell order for plain SKI (opts.keep_points): {t_1..t_d, y} records and cell keys
    void *pts;
    uint32_t *pkeys;
    // solver workspace (owned)
    fk::SolveWork *work;
    // rank-k predictive-covariance factor (owned): R = K (P_hat + W^T b d^T) L^{-T}, m x k FP64
    // row-major, for the kernel it was built with
    double *lowrank;
    int lowrank_k;      // Lanczos steps taken (fewer than requested if the Krylov space closed)
    int lowrank_kreq;   // steps requested
    fkski_kernel lowrank_kern;
};

namespace fk {
// Implemented in the respective translation units.
int precompute_impl(const fkski_grid *grid, const void *X, const void *y, const void *Z, int64_t n,
                    int dtype, const fkski_opts *opts, fkski_stats **out, cudaStream_t s);
int kg_mvm_impl(const fkski_grid *grid, const fkski_kernel *kern, int param, const void *v, void *out,
                int nrhs, int dtype, cudaStream_t s);
int kg_mvm_noalloc_impl(const fkski_grid *grid, const fkski_kernel *kern, int param, const void *v, void *out,
                        int nrhs, int dtype, cudaStream_t s);
int band_mvm_impl(const fkski_stats *st, const void *x, void *u, int nrhs, int dtype, cudaStream_t s);
int stats_band_as(fkski_stats *st, int dtype, const void **band, const void **wty, const void **wtz,
                  cudaStream_t s);
int solve_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, void *a_out,
               void *v_out, fkski_info *info, cudaStream_t s);
int predict_impl(const fkski_stats *st, const void *v, int vdtype, const void *Xs, int xdtype,
                 int64_t ns, void *mu, cudaStream_t s);
int posterior_cov_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, const void *Xs, int xdtype,
                       int64_t ns, double *cov, fkski_info *info, cudaStream_t s);
int posterior_cov_lowrank_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, int k,
                               const void *Xs, int xdtype, int64_t ns, double *cov, fkski_info *info, cudaStream_t s);
int ski_solve_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, void *a_out, void *v_out,
                   fkski_info *info, cudaStream_t s);
int efla_probe_tridiag(fkski_stats *st, const fkski_kernel *kern, int k, int probe, std::vector<double> &dg,
                       std::vector<double> &of, fkski_info *info, cudaStream_t s);
int logdet_lanczos_impl(fkski_stats *st, const fkski_kernel *kern, int k, double *logdet, double *terms,
                        fkski_info *info, cudaStream_t s);
int solve_batched_impl(int P, fkski_stats *const *sts, const fkski_kernel *kernels, const fkski_opts *opts,
                       void *const *a_out, void *const *v_out, fkski_info *info, cudaStream_t s);
int predict_batched_impl(int P, const fkski_stats *const *st, const void *const *v, int vdtype, const void *const *Xs,
                         int xdtype, const int64_t *ns, void *const *mu, int *status, cudaStream_t s);
int loglik_forward_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts,
                        double *L, fkski_info *info, cudaStream_t s);
int loglik_backward_impl(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts,
                         double *grad, fkski_info *info, cudaStream_t s);
void free_solve_work(SolveWork *w);

// K_G operator objects (kg.cu), used by the solvers.
struct KgOp;
int kgop_create(const fkski_grid *grid, int dtype, KgOp **op);
void kgop_destroy(KgOp *op);
// Recompute spectra for the hyperparameters (param as in fkski_kg_mvm).
int kgop_set(KgOp *op, const fkski_kernel *kern, int param, cudaStream_t s);
// out = K v (or dK v) for nrhs vectors; if addv != nullptr: out = K v + alpha * addv
// (addv has the same layout as v).  Scratch grows on demand (see kgop_reserve).
int kgop_apply(KgOp *op, const void *v, void *out, int nrhs, const void *addv, double alpha,
               cudaStream_t s);
// Pre-allocate the scratch for nrhs vectors (call before capturing applications in a graph).
int kgop_reserve(KgOp *op, int nrhs);
// Time the launch configurations of this operator's passes for nrhs vectors (RBF) and keep the
// fastest per pass shape; needs the spectra (kgop_set).  Not inside a stream capture.
int kgop_tune(KgOp *op, int nrhs, cudaStream_t s);
// Text table of the tuned pass shapes (returns the size needed including the terminator).
size_t kg_tuning_table(char *buf, size_t len);
// Same, with alpha read from device memory (a double) so graphs can be reused.
// Device flag that makes every kernel of later products return at once while it is set (null: none).
void kgop_set_gate(KgOp *op, const int *gate);
int kgop_apply_dev(KgOp *op, const void *v, void *out, int nrhs, const void *addv,
                   const double *alpha_dev, cudaStream_t s);
}  // namespace fk

// ------------------------------------------------------------------ device helpers
namespace fk {

// Exact float sequence for the cell of one FP32 coordinate (TwoSum + FMA product); returns
// 0 inside, 1 outside [1, M-2], 2 non-finite.  Every operation is an explicit round-to-nearest
// intrinsic so the compiler cannot contract or reorder it.
__device__ __forceinline__ int axis_cell_f32(float x, const AxisKeyF &k, int &cell, float &t) {
    if (!isfinite(x)) return 2;
    const float a = x, b = -k.L1;
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    e = __fsub_rn(e, k.L2);
    const float d1 = __fadd_rn(s, e);
    const float d2 = __fsub_rn(e, __fsub_rn(d1, s));
    const float p = __fmul_rn(d1, k.I1);
    float q = __fmaf_rn(d1, k.I1, -p);
    q = __fmaf_rn(d1, k.I2, q);
    q = __fmaf_rn(d2, k.I1, q);
    const float s1 = __fadd_rn(p, q);
    const float s2 = __fsub_rn(q, __fsub_rn(s1, p));
    const bool in_lo = (s1 > 1.0f) || (s1 == 1.0f && s2 >= 0.0f);
    const bool in_hi = (s1 < k.top) || (s1 == k.top && s2 <= 0.0f);
    if (!(in_lo && in_hi)) return 1;
    float c = floorf(s1);
    if (s1 == c && s2 < 0.0f) c = __fsub_rn(c, 1.0f);
    int ci = (int)c;
    ci = ci < 1 ? 1 : (ci > k.M - 3 ? k.M - 3 : ci);
    t = __fadd_rn(__fsub_rn(s1, (float)ci), s2);
    cell = ci;
    return 0;
}

__device__ __forceinline__ int axis_cell_f64(double x, const AxisKeyD &k, int &cell, double &t) {
    if (!isfinite(x)) return 2;
    const double s = __dmul_rn(__dsub_rn(x, k.lo), k.ih);
    if (!(s >= 1.0 && s <= (double)(k.M - 2))) return 1;
    int ci = (int)floor(s);
    ci = ci < 1 ? 1 : (ci > k.M - 3 ? k.M - 3 : ci);
    t = __dsub_rn(s, (double)ci);
    cell = ci;
    return 0;
}

template <typename T>
__device__ __forceinline__ int axis_cell(T x, const KeyParams &kp, int k, int &cell, T &t);
template <>
__device__ __forceinline__ int axis_cell<float>(float x, const KeyParams &kp, int k, int &cell, float &t) {
    return axis_cell_f32(x, kp.f[k], cell, t);
}
template <>
__device__ __forceinline__ int axis_cell<double>(double x, const KeyParams &kp, int k, int &cell, double &t) {
    return axis_cell_f64(x, kp.g[k], cell, t);
}

// Point record: local cell coordinates t_1..t_d (unused axes 0) and the target y.
template <typename T>
struct alignas(4 * sizeof(T)) Rec4 {
    T t[3];
    T y;
};

// Cubic-convolution weights (Keys, a = -1/2) on nodes c-1..c+2 written in the cubic Bernstein
// basis, which has no cancellation on [0, 1]:
//   w0 = -1/2 t u^2, w1 = u^3 + 3 t u^2 + 1/2 t^2 u, w2 = 1/2 t u^2 + 3 t^2 u + t^3,
//   w3 = -1/2 t^2 u,  u = 1 - t.
template <typename T>
__device__ __forceinline__ void keys_weights(T t, T w[4]) {
    const T u = T(1) - t;
    const T tu2 = t * u * u, t2u = t * t * u;
    w[0] = T(-0.5) * tu2;
    w[1] = u * u * u + T(3) * tu2 + T(0.5) * t2u;
    w[2] = T(0.5) * tu2 + T(3) * t2u + t * t * t;
    w[3] = T(-0.5) * t2u;
}

// Degree-6 Bernstein basis B_p(t) = C(6,p) t^p (1-t)^(6-p), p = 0..6.
template <typename T>
__device__ __forceinline__ void bern6(T t, T b[7]) {
    const T u = T(1) - t;
    const T t2 = t * t, t3 = t2 * t, u2 = u * u, u3 = u2 * u;
    b[0] = u3 * u3;
    b[1] = T(6) * t * u2 * u3;
    b[2] = T(15) * t2 * u2 * u2;
    b[3] = T(20) * t3 * u3;
    b[4] = T(15) * t2 * t2 * u2;
    b[5] = T(6) * t2 * t3 * u;
    b[6] = t3 * t3;
}

// SplitMix64 output k of the stream started at `seed` (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Rademacher probe sign z_p(i) in {-1, +1}: counter k = p * 2^40 + i + 1.
template <typename T>
__device__ __forceinline__ T rademacher(uint64_t seed, int p, int64_t i) {
    const uint64_t k = ((uint64_t)p << 40) + (uint64_t)i + 1ULL;
    return (splitmix64_at(seed, k) >> 63) ? T(-1) : T(1);
}

}  // namespace fk
