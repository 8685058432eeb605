// C ABI of libfkski.so (declared in include/fkski.h): argument checks, stream plumbing, the stats
// object's lifetime, export and save/load.  All compute lives in the other translation units.
#include "fkski_internal.cuh"

#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

namespace fk {

void destroy_stats(fkski_stats *st) {
    if (!st) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (st->device != cur) cudaSetDevice(st->device);
    free_solve_work(st->work);
    void *ptrs[] = {st->band_alt, st->wty_alt, st->wtz_alt, st->wty_df, st->wtz_df, st->keys, st->perm, st->offsets,
                    st->lowrank, st->pts, st->pkeys};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    // pool blocks: once the device is idle (cudaFree above already waited for it when it ran),
    // hand them back to the pool
    cudaDeviceSynchronize();
    void *pooled[] = {st->band, st->wty, st->wtz};
    for (void *p : pooled)
        if (p) cudaFreeAsync(p, 0);
    if (st->device != cur) cudaSetDevice(cur);
    delete st;
}

static cudaStream_t S(void *stream) { return reinterpret_cast<cudaStream_t>(stream); }

static thread_local char g_detail[256] = "";
static std::atomic<long long> g_launches{0};

void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Library memory pool per device for stream-ordered temporaries (precompute scratch and the
// like): freed blocks stay cached in the pool (release threshold: unlimited), so repeated calls
// of the same size map no new memory.  fkski_trim_memory() hands the cache back.
static std::mutex g_pool_mu;
static constexpr int kMaxDevices = 64;
static cudaMemPool_t g_pool[kMaxDevices];

static cudaError_t pool_for(int dev, cudaMemPool_t *out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;  // beyond the pool table
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t thr = UINT64_MAX;
        e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr);
        if (e != cudaSuccess) return e;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

static std::mutex g_attr_mu;
static std::map<std::pair<int, const void *>, size_t> g_attr;

int raise_smem_limit(const void *func, size_t bytes) {
    int dev = 0;
    FK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_attr_mu);
    size_t &cur = g_attr[std::make_pair(dev, func)];
    if (bytes <= cur) return FKSKI_OK;
    FK_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return FKSKI_OK;
}

int pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    int dev = 0;
    FK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return FKSKI_E_UNSUPPORTED;
    cudaMemPool_t pool;
    FK_CUDA(pool_for(dev, &pool));
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s);
    if (e == cudaErrorMemoryAllocation) {  // give the cached blocks back and try once more
        cudaGetLastError();
        cudaStreamSynchronize(s);
        cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return note_cuda_error(e, __FILE__, __LINE__);
    }
    return FKSKI_OK;
}

int note_cuda_error(cudaError_t e, const char *file, int line) {
    const char *base = strrchr(file, '/');
    snprintf(g_detail, sizeof(g_detail), "%s (%d) at %s:%d", cudaGetErrorString(e), (int)e, base ? base + 1 : file,
             line);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FKSKI_E_OOM : FKSKI_E_CUDA;
}

}  // namespace fk

using namespace fk;

extern "C" {

void fkski_default_opts(fkski_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->rtol = 1e-6;
    o->maxiter = 1000;
    o->x0_mode = FKSKI_X0_Y_OVER_S2;
    o->precision = FKSKI_MIXED;
    o->check_every = 16;
    o->n_probes = 0;
    o->probe_seed = 0;
    o->iterate_budget_bytes = (size_t)1 << 30;
    o->keep_sort = 0;
}

const char *fkski_strerror(int st) {
    switch (st) {
        case FKSKI_OK: return "ok";
        case FKSKI_E_INVALID_ARG: return "invalid argument";
        case FKSKI_E_OUT_OF_GRID: return "point outside the grid interior [1, M-2]";
        case FKSKI_E_NONFINITE: return "non-finite input";
        case FKSKI_E_NOT_CONVERGED: return "CG did not converge within maxiter";
        case FKSKI_E_BREAKDOWN: return "CG breakdown (non-positive curvature or non-finite inner product)";
        case FKSKI_E_TIMEOUT: return "bounded device wait gave up";
        case FKSKI_E_OOM: return "device out of memory";
        case FKSKI_E_CUDA: return "CUDA runtime error";
        case FKSKI_E_UNSUPPORTED: return "size not supported by this build";
        case FKSKI_E_IO: return "file error";
        default: return "unknown status";
    }
}

const char *fkski_last_error_detail(void) { return g_detail; }

size_t fkski_tuning_table(char *buf, size_t len) { return kg_tuning_table(buf, len); }

long long fkski_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int fkski_trim_memory(void) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    for (int d = 0; d < kMaxDevices; ++d)
        if (g_pool[d] && cudaMemPoolTrimTo(g_pool[d], 0) != cudaSuccess) return note_cuda_error(cudaGetLastError(), __FILE__, __LINE__);
    return FKSKI_OK;
}

int fkski_precompute(const fkski_grid *grid, const void *X, const void *y, const void *Z, int64_t n, int dtype,
                     const fkski_opts *opts, fkski_stats **out, void *stream) {
    return precompute_impl(grid, X, y, Z, n, dtype, opts, out, S(stream));
}

int fkski_stats_info(const fkski_stats *st, fkski_grid *grid, int64_t *n, int64_t *m, int64_t *ncells, int *n_probes,
                     double *yty, int *dtype) {
    if (!st) return FKSKI_E_INVALID_ARG;
    if (grid) *grid = st->grid;
    if (n) *n = st->n;
    if (m) *m = st->m;
    if (ncells) *ncells = st->ncells;
    if (n_probes) *n_probes = st->nprobes;
    if (yty) *yty = st->yty;
    if (dtype) *dtype = st->dtype;
    return FKSKI_OK;
}

static int copy_to_host_f64(const void *src, int dtype, int64_t count, double *dst, cudaStream_t s) {
    if (!dst || count == 0) return FKSKI_OK;
    if (dtype == FKSKI_F64) {
        FK_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
        FK_CUDA(cudaStreamSynchronize(s));
        return FKSKI_OK;
    }
    std::vector<float> tmp((size_t)count);
    FK_CUDA(cudaMemcpyAsync(tmp.data(), src, sizeof(float) * count, cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < count; ++i) dst[i] = (double)tmp[(size_t)i];
    return FKSKI_OK;
}

int fkski_stats_export(const fkski_stats *st, double *band, double *wty, double *wtz, double *ztz, void *stream) {
    if (!st) return FKSKI_E_INVALID_ARG;
    const cudaStream_t s = S(stream);
    FK_TRY(copy_to_host_f64(st->band, st->dtype, ipow(7, st->d) * st->m, band, s));
    FK_TRY(copy_to_host_f64(st->wty, st->dtype, st->m, wty, s));
    if (st->nprobes > 0) FK_TRY(copy_to_host_f64(st->wtz, st->dtype, st->nprobes * st->m, wtz, s));
    if (ztz)
        for (int p = 0; p < st->nprobes; ++p) ztz[p] = st->ztz[p];
    return FKSKI_OK;
}

int fkski_stats_export_sort(const fkski_stats *st, uint32_t *keys, int64_t *perm, int64_t *offsets, void *stream) {
    if (!st) return FKSKI_E_INVALID_ARG;
    if (!st->keys || !st->perm || !st->offsets) return FKSKI_E_UNSUPPORTED;
    const cudaStream_t s = S(stream);
    if (keys) FK_CUDA(cudaMemcpyAsync(keys, st->keys, sizeof(uint32_t) * st->n, cudaMemcpyDeviceToHost, s));
    std::vector<uint32_t> tmp;
    if (perm) {
        tmp.resize((size_t)st->n);
        FK_CUDA(cudaMemcpyAsync(tmp.data(), st->perm, sizeof(uint32_t) * st->n, cudaMemcpyDeviceToHost, s));
        FK_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < st->n; ++i) perm[i] = tmp[(size_t)i];
    }
    if (offsets) {
        tmp.resize((size_t)(st->ncells + 1));
        FK_CUDA(cudaMemcpyAsync(tmp.data(), st->offsets, sizeof(uint32_t) * (st->ncells + 1), cudaMemcpyDeviceToHost, s));
        FK_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i <= st->ncells; ++i) offsets[i] = tmp[(size_t)i];
    }
    FK_CUDA(cudaStreamSynchronize(s));
    return FKSKI_OK;
}

// File layout: magic "FKSKI01\0", then the fixed header, then band, wty, wtz in the stats dtype.
struct SaveHeader {
    char magic[8];
    fkski_grid grid;
    int32_t d, dtype, nprobes, pad;
    int64_t n, m, ncells;
    uint64_t seed;
    double yty;
    double ztz[kMaxProbes];
};

int fkski_stats_save(const fkski_stats *st, const char *path, void *stream) {
    if (!st || !path) return FKSKI_E_INVALID_ARG;
    const cudaStream_t s = S(stream);
    SaveHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "FKSKI01", 8);
    h.grid = st->grid;
    h.d = st->d;
    h.dtype = st->dtype;
    h.nprobes = st->nprobes;
    h.n = st->n;
    h.m = st->m;
    h.ncells = st->ncells;
    h.seed = st->probe_seed;
    h.yty = st->yty;
    for (int p = 0; p < kMaxProbes; ++p) h.ztz[p] = st->ztz[p];
    const size_t es = st->dtype == FKSKI_F32 ? 4 : 8;
    const size_t nb = (size_t)ipow(7, st->d) * st->m;
    std::vector<char> buf(es * (nb + st->m + (size_t)st->nprobes * st->m));
    FK_CUDA(cudaMemcpyAsync(buf.data(), st->band, es * nb, cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaMemcpyAsync(buf.data() + es * nb, st->wty, es * st->m, cudaMemcpyDeviceToHost, s));
    if (st->nprobes)
        FK_CUDA(cudaMemcpyAsync(buf.data() + es * (nb + st->m), st->wtz, es * st->nprobes * st->m, cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaStreamSynchronize(s));
    FILE *f = fopen(path, "wb");
    if (!f) return FKSKI_E_IO;
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? FKSKI_OK : FKSKI_E_IO;
}

int fkski_stats_load(const char *path, fkski_stats **out, void *stream) {
    if (!path || !out) return FKSKI_E_INVALID_ARG;
    *out = nullptr;
    const cudaStream_t s = S(stream);
    FILE *f = fopen(path, "rb");
    if (!f) return FKSKI_E_IO;
    SaveHeader h;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, "FKSKI01", 8) != 0 || h.d < 1 || h.d > 3 ||
        (h.dtype != FKSKI_F32 && h.dtype != FKSKI_F64) || h.nprobes < 0 || h.nprobes > kMaxProbes || h.m < 1) {
        fclose(f);
        return FKSKI_E_IO;
    }
    const size_t es = h.dtype == FKSKI_F32 ? 4 : 8;
    const size_t nb = (size_t)ipow(7, h.d) * h.m;
    std::vector<char> buf(es * (nb + h.m + (size_t)h.nprobes * h.m));
    const bool ok = fread(buf.data(), 1, buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return FKSKI_E_IO;
    fkski_stats *st = new fkski_stats;
    memset(st, 0, sizeof(*st));
    st->grid = h.grid;
    st->d = h.d;
    st->dtype = h.dtype;
    st->n = h.n;
    st->m = h.m;
    st->ncells = h.ncells;
    st->nprobes = h.nprobes;
    st->probe_seed = h.seed;
    st->yty = h.yty;
    for (int p = 0; p < kMaxProbes; ++p) st->ztz[p] = h.ztz[p];
    cudaGetDevice(&st->device);
    int rc = FKSKI_OK;
    if (pool_alloc(&st->band, es * nb, s) != FKSKI_OK || pool_alloc(&st->wty, es * h.m, s) != FKSKI_OK ||
        (h.nprobes && pool_alloc(&st->wtz, es * h.nprobes * h.m, s) != FKSKI_OK))
        rc = FKSKI_E_OOM;
    if (rc == FKSKI_OK) {
        if (cudaMemcpyAsync(st->band, buf.data(), es * nb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(st->wty, buf.data() + es * nb, es * h.m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            (h.nprobes && cudaMemcpyAsync(st->wtz, buf.data() + es * (nb + h.m), es * h.nprobes * h.m,
                                          cudaMemcpyHostToDevice, s) != cudaSuccess) ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = FKSKI_E_CUDA;
    }
    if (rc != FKSKI_OK) {
        destroy_stats(st);
        return rc;
    }
    *out = st;
    return FKSKI_OK;
}

void fkski_destroy(fkski_stats *st) { destroy_stats(st); }

int fkski_kg_mvm(const fkski_grid *grid, const fkski_kernel *kern, int param, const void *v, void *out, int nrhs,
                 int dtype, void *stream) {
    return kg_mvm_impl(grid, kern, param, v, out, nrhs, dtype, S(stream));
}

int fkski_kg_mvm_noalloc(const fkski_grid *grid, const fkski_kernel *kern, int param, const void *v, void *out,
                         int nrhs, int dtype, void *stream) {
    return kg_mvm_noalloc_impl(grid, kern, param, v, out, nrhs, dtype, S(stream));
}

int fkski_band_mvm(const fkski_stats *st, const void *x, void *u, int nrhs, int dtype, void *stream) {
    return band_mvm_impl(st, x, u, nrhs, dtype, S(stream));
}

int fkski_solve(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, void *a_out, void *v_out,
                fkski_info *info, void *stream) {
    return solve_impl(st, kern, opts, a_out, v_out, info, S(stream));
}

int fkski_logdet_lanczos(fkski_stats *st, const fkski_kernel *kern, int k, double *logdet_out, double *terms,
                         fkski_info *info, void *stream) {
    return logdet_lanczos_impl(st, kern, k, logdet_out, terms, info, S(stream));
}

int fkski_ski_solve(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, void *a_out, void *v_out,
                    fkski_info *info, void *stream) {
    return ski_solve_impl(st, kern, opts, a_out, v_out, info, S(stream));
}

int fkski_posterior_cov(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, const void *Xstar, int xdtype,
                        int64_t nstar, double *cov_out, fkski_info *info, void *stream) {
    return posterior_cov_impl(st, kern, opts, Xstar, xdtype, nstar, cov_out, info, S(stream));
}

int fkski_posterior_cov_lowrank(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, int k,
                                const void *Xstar, int xdtype, int64_t nstar, double *cov_out, fkski_info *info,
                                void *stream) {
    return posterior_cov_lowrank_impl(st, kern, opts, k, Xstar, xdtype, nstar, cov_out, info, S(stream));
}

int fkski_precompute_batched(int nprob, const fkski_grid *grids, const void *const *X, const void *const *y,
                             const int64_t *n, int dtype, const fkski_opts *opts, fkski_stats **out, void *stream) {
    if (nprob < 1 || !grids || !X || !y || !n || !out) return FKSKI_E_INVALID_ARG;
    for (int p = 0; p < nprob; ++p) out[p] = nullptr;
    for (int p = 0; p < nprob; ++p) {
        const int rc = fkski_precompute(&grids[p], X[p], y[p], nullptr, n[p], dtype, opts, &out[p], stream);
        if (rc != FKSKI_OK) {
            for (int q = 0; q < p; ++q) {
                fkski_destroy(out[q]);
                out[q] = nullptr;
            }
            out[p] = nullptr;
            return rc;
        }
    }
    return FKSKI_OK;
}

int fkski_solve_batched(int nprob, fkski_stats *const *st, const fkski_kernel *kernels, const fkski_opts *opts,
                        void *const *a_out, void *const *v_out, fkski_info *info, void *stream) {
    return solve_batched_impl(nprob, st, kernels, opts, a_out, v_out, info, S(stream));
}

int fkski_predict_batched(int nprob, const fkski_stats *const *st, const void *const *v, int vdtype,
                          const void *const *Xstar, int xdtype, const int64_t *nstar, void *const *mu_out, int *status,
                          void *stream) {
    return predict_batched_impl(nprob, st, v, vdtype, Xstar, xdtype, nstar, mu_out, status, S(stream));
}

int fkski_predict(const fkski_stats *st, const void *v, int vdtype, const void *Xstar, int xdtype, int64_t nstar,
                  void *mu_out, void *stream) {
    return predict_impl(st, v, vdtype, Xstar, xdtype, nstar, mu_out, S(stream));
}

int fkski_loglik_forward(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, double *loglik_out,
                         fkski_info *info, void *stream) {
    return loglik_forward_impl(st, kern, opts, loglik_out, info, S(stream));
}

int fkski_loglik_backward(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, double *grad_out,
                          fkski_info *info, void *stream) {
    return loglik_backward_impl(st, kern, opts, grad_out, info, S(stream));
}

int fkski_grad(fkski_stats *st, const fkski_kernel *kern, const fkski_opts *opts, double *loglik_out,
               double *grad_out, fkski_info *info, void *stream) {
    fkski_opts o;
    if (opts) o = *opts; else fkski_default_opts(&o);
    o.iterate_budget_bytes = (size_t)-1;
    double L = 0.0;
    int rc = loglik_forward_impl(st, kern, &o, &L, info, S(stream));
    if (rc != FKSKI_OK && rc != FKSKI_E_NOT_CONVERGED) return rc;
    if (loglik_out) *loglik_out = L;
    const int rb = loglik_backward_impl(st, kern, &o, grad_out, nullptr, S(stream));
    return rb != FKSKI_OK ? rb : rc;
}

}  // extern "C"
