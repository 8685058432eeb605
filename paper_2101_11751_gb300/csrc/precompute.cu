// Sufficient-statistics precompute (Sec. 3.1): W^T W as 7^d diagonals (Claim 2), W^T y, y^T y,
// W^T z_p and z_p^T z_p for probes -- one O(n) pass over the points plus O(m) band assembly.
//
// Pipeline (all on one stream):
//   k_keys          cell index per point (exact float sequence), local coords t, per-cell counts
//   scan            counts -> segment offsets
//   radix passes    stable LSD sort of (cell key, point index) -> permutation
//   k_moments       per cell: degree-6 Bernstein moments  M[p] = sum_i prod_k B_{p_k}(t_ik)
//                   (7^d values) and Y[a] = sum_i y_i prod_k w_{a_k}(t_ik) (4^d values), in sorted
//                   order (deterministic), then the last-axis contraction to grid nodes
//   k_axis_pass     the remaining per-axis contractions -> band (7^d x m) and W^T y
//   k_probe_moments / passes   W^T z_p for the probes
//
// Why moments: each 1-D product w_a(t) w_b(t) of cubic-convolution weights is a polynomial of
// degree 6, so the 4^d x 4^d block sum_i w_i w_i^T of a cell is a fixed linear image of the 7^d
// moments (Claim 2 bounds the block by (2r)^(2d) = 4096 products per point in 3-D; the moments
// need 343).  In the Bernstein basis every product has coefficients of one sign, so the
// expansion has no cancellation.  The band entry (W^T W)[j, j+delta] collects, per axis, the
// cells c = j - a (a = 0..3) that contain both nodes; this is separable across axes.
#include "fkski_internal.cuh"

#include <algorithm>
#include <type_traits>
#include <utility>
#include <vector>

namespace fk {

// ------------------------------------------------------------------ host: key constants
static void split_double(double v, float *hi, float *lo) {
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
}

KeyParams make_key_params(const fkski_grid &g) {
    KeyParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.d = g.d;
    int64_t stride = 1;
    for (int k = g.d - 1; k >= 0; --k) {
        kp.ncell[k] = g.M[k] - 3;
        kp.cstride[k] = stride;
        stride *= g.M[k] - 3;
    }
    for (int k = 0; k < g.d; ++k) {
        split_double(g.lo[k], &kp.f[k].L1, &kp.f[k].L2);
        split_double(1.0 / g.h[k], &kp.f[k].I1, &kp.f[k].I2);
        kp.f[k].top = (float)(g.M[k] - 2);
        kp.f[k].M = (int)g.M[k];
        kp.g[k].lo = g.lo[k];
        kp.g[k].ih = 1.0 / g.h[k];
        kp.g[k].M = (int)g.M[k];
    }
    return kp;
}

// Bernstein coefficients of the products w_a w_b (a, b = 0..3) in the degree-6 basis:
// with w_a = sum_q beta_a[q] B3_q, B3_q B3_r = C(3,q) C(3,r) / C(6,q+r) B6_{q+r}.
// Table E[a][delta+3][p] = coefficient of B6_p in w_a w_{a+delta} (0 if a+delta is off-stencil),
// as a constexpr function: with compile-time arguments (the contraction helpers below) it folds
// to a literal, and the kernels skip the 64 of its 112 on-stencil entries that are zero.
__host__ __device__ constexpr double etab_coef(int a, int dl, int p) {
    constexpr double beta[4][4] = {{0, -1.0 / 6, 0, 0}, {1, 1, 1.0 / 6, 0}, {0, 1.0 / 6, 1, 1}, {0, 0, -1.0 / 6, 0}};
    constexpr double c3[4] = {1, 3, 3, 1};
    constexpr double c6[7] = {1, 6, 15, 20, 15, 6, 1};
    const int b = a + dl - 3;
    double v = 0.0;
    if (b >= 0 && b < 4)
        for (int q = 0; q < 4; ++q) {
            const int r = p - q;
            if (r >= 0 && r < 4) v += beta[a][q] * beta[b][r] * c3[q] * c3[r] / c6[p];
        }
    return v;
}

// acc[dl] += sum_p E[A][dl][p] v[p] for every dl, p in increasing order, the entries as
// compile-time constants (zero entries, including the off-stencil dl, emit nothing).
template <int A, int DL, int P, typename T>
__device__ __forceinline__ void etab_term(T &acc, T v) {
    constexpr double c = etab_coef(A, DL, P);
    if constexpr (c != 0.0) acc = fma((T)c, v, acc);
}
template <int A, typename T, int... I>
__device__ __forceinline__ void etab_accumulate_seq(T (&acc)[7], const T *v, std::integer_sequence<int, I...>) {
    (etab_term<A, I / 7, I % 7>(acc[I / 7], v[I % 7]), ...);
}
template <int A, typename T>
__device__ __forceinline__ void etab_accumulate(T (&acc)[7], const T *v) {
    etab_accumulate_seq<A>(acc, v, std::make_integer_sequence<int, 49>{});
}


// Points in cell order for plain SKI: pts[k] = rec[perm[k]], pkeys[k] = keys[perm[k]].
template <typename T>
__global__ void k_gather_points(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ keys,
                                const Rec4<T> *__restrict__ rec, int64_t n, Rec4<T> *__restrict__ pts,
                                uint32_t *__restrict__ pkeys) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = perm[k];
        pts[k] = rec[i];
        pkeys[k] = keys[i];
    }
}

// ------------------------------------------------------------------ K1: cell keys
// One thread per point (uniform trip count per block so warp collectives stay converged).
// Writes key[i], rec[i] = (t_1..t_d, y_i), adds to the per-cell counts (warp-aggregated
// integer atomics: exact) and accumulates y^2 (FP32 runs of 8, FP64 across) per block.
// Blocks walk whole radix tiles (RS_TILE consecutive points) so that the first radix pass's
// per-tile digit histogram (digit = key & (2^hbits - 1)) is counted here too and written in the
// layout k_radix_hist would write (digit-major, ghist[digit * ntiles + tile]).  A point that
// fails its checks is written with key 0 and counted under digit 0, as the sort will see it.
constexpr int RS_T = 256;
constexpr int RS_ITEMS = 32;
constexpr int RS_TILE = RS_T * RS_ITEMS;  // 8192; each warp owns 1024 contiguous keys
constexpr int RS_MAXBITS = 10;

template <typename T, int D>
__global__ void __launch_bounds__(RS_T) k_keys(const T *__restrict__ X, const T *__restrict__ y, int64_t n,
                                               KeyParams kp, uint32_t *__restrict__ keys,
                                               Rec4<T> *__restrict__ rec, uint32_t *__restrict__ counts,
                                               double *__restrict__ ypart, int *__restrict__ status,
                                               uint32_t *__restrict__ ghist, int hbits, int64_t ntiles) {
    __shared__ uint32_t hist[1 << RS_MAXBITS];
    const int lane = threadIdx.x & 31;
    const int nb = 1 << hbits;
    const uint32_t hmask = (uint32_t)nb - 1u;
    double ysq = 0.0;
    float run = 0.f;
    int nrun = 0;
    int bad = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < nb; i += RS_T) hist[i] = 0u;
        __syncthreads();
        for (int k = 0; k < RS_ITEMS; ++k) {
            const int64_t i = tile * RS_TILE + (int64_t)k * RS_T + threadIdx.x;
            uint32_t key = 0xFFFFFFFFu;
            bool failed = false;
            if (i < n) {
                Rec4<T> r;
                r.t[0] = r.t[1] = r.t[2] = T(0);
                int64_t kk = 0;
                int st = 0;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    int c = 1;
                    T t = T(0);
                    const int sk = axis_cell<T>(X[(int64_t)a * n + i], kp, a, c, t);
                    st |= sk;
                    kk += (int64_t)(c - 1) * kp.cstride[a];
                    r.t[a] = t;
                }
                const T yi = y[i];
                if (!isfinite((double)yi)) st |= 2;
                if (st == 0) {
                    key = (uint32_t)kk;
                    r.y = yi;
                    rec[i] = r;
                    keys[i] = key;
                    if (sizeof(T) == 4) {
                        const float yf = (float)yi;
                        run = fmaf(yf, yf, run);
                        if (++nrun == 8) { ysq += (double)run; run = 0.f; nrun = 0; }
                    } else {
                        ysq += (double)yi * (double)yi;
                    }
                } else {
                    bad |= (st & 2) ? ST_NONFINITE : ST_OUT_OF_GRID;
                    failed = true;
                    keys[i] = 0;
                    r.y = T(0);
                    rec[i] = r;
                }
            }
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
            if (key != 0xFFFFFFFFu && lane == __ffs(peers) - 1) {
                atomicAdd(&counts[key], (uint32_t)__popc(peers));
                if (ghist) atomicAdd(&hist[key & hmask], (uint32_t)__popc(peers));
            }
            if (failed && ghist) atomicAdd(&hist[0], 1u);
        }
        __syncthreads();
        if (ghist)
            for (int d = threadIdx.x; d < nb; d += RS_T) ghist[(int64_t)d * ntiles + tile] = hist[d];
        __syncthreads();
    }
    ysq += (double)run;
    if (bad) atomicOr(status, bad);
    // block reduce ysq in FP64 (fixed order)
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ysq += __shfl_xor_sync(0xFFFFFFFFu, ysq, o);
    if (lane == 0) sh[threadIdx.x >> 5] = ysq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        ypart[blockIdx.x] = s;
    }
}

// Sum of `np` FP64 partials in index order (one thread): deterministic.
__global__ void k_sum_partials(const double *__restrict__ part, int np, int nvec, double *__restrict__ out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvec) return;
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[(int64_t)i * nvec + v];
    out[v] = s;
}

// Sum of squares of each of `nvec` rows (length n) of Z: per block FP64 partials.
template <typename T>
__global__ void k_rowsq_partials(const T *__restrict__ Z, int64_t n, int nvec, double *__restrict__ part,
                                 int *__restrict__ status) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31;
    for (int v = 0; v < nvec; ++v) {
        double acc = 0.0;
        int bad = 0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const double z = (double)Z[(int64_t)v * n + i];
            if (!isfinite(z)) bad = 1;
            acc += z * z;
        }
        if (bad) atomicOr(status, ST_NONFINITE);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
            part[(int64_t)blockIdx.x * nvec + v] = s;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ exclusive scan (u32)
constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *sh, uint32_t &total) {
    // sh: 32 words
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    const uint32_t before = w > 0 ? sh[w - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                                                        uint32_t *__restrict__ bsum) {
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + (int64_t)k * SCAN_T + threadIdx.x;
        if (i < n) s += in[i];
    }
    uint32_t tot;
    block_exclusive_scan(s, sh, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Exclusive scan of the block sums in one block (sequential over chunks of 256).
__global__ void __launch_bounds__(SCAN_T) k_scan_top(uint32_t *__restrict__ bsum, int64_t nb, uint32_t *__restrict__ total_out) {
    __shared__ uint32_t sh[32];
    uint32_t carry = 0;
    for (int64_t c = 0; c < nb; c += SCAN_T) {
        const int64_t i = c + threadIdx.x;
        const uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, sh, tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_down(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                      int64_t n, const uint32_t *__restrict__ bsum) {
    __shared__ uint32_t sh[32];
    __shared__ uint32_t vals[SCAN_TILE];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + (int64_t)k * SCAN_T + threadIdx.x;
        vals[k * SCAN_T + threadIdx.x] = i < n ? in[i] : 0u;
    }
    __syncthreads();
    // each thread owns SCAN_ITEMS consecutive values
    uint32_t loc[SCAN_ITEMS];
    uint32_t s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        loc[k] = vals[threadIdx.x * SCAN_ITEMS + k];
        s += loc[k];
    }
    uint32_t tot;
    uint32_t ex = block_exclusive_scan(s, sh, tot) + bsum[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        vals[threadIdx.x * SCAN_ITEMS + k] = ex;
        ex += loc[k];
    }
    __syncthreads();
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + (int64_t)k * SCAN_T + threadIdx.x;
        if (i < n) out[i] = vals[k * SCAN_T + threadIdx.x];
    }
}

// Exclusive scan of n u32 values (in may equal out); writes the total to out[n] if with_total.
static int exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, bool with_total, uint32_t *bsum,
                              cudaStream_t s) {
    const int64_t nb = cdiv(n, SCAN_TILE);
    k_scan_reduce<<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, bsum);
    FK_LAUNCH();
    k_scan_top<<<1, SCAN_T, 0, s>>>(bsum, nb, with_total ? out + n : nullptr);
    FK_LAUNCH();
    k_scan_down<<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, n, bsum);
    FK_LAUNCH();
    return FKSKI_OK;
}

// ------------------------------------------------------------------ stable LSD radix sort

// Lanes of the warp holding the same digit (lanes outside `valid_mask` never match).
__device__ __forceinline__ unsigned digit_peers(uint32_t dg, int bits, unsigned valid_mask) {
    (void)bits;
    return __match_any_sync(0xFFFFFFFFu, dg) & valid_mask;
}

// Key of element i of a pass input: the cell keys themselves (first pass) or the .x half of the
// packed (key, point index) pairs an earlier pass wrote.
template <bool PACKED, typename I>
__device__ __forceinline__ uint32_t rs_key(const uint32_t *__restrict__ kin, I i) {
    return PACKED ? __ldcs(kin + 2 * i) : __ldcs(kin + i);
}

template <bool PACKED>
__global__ void __launch_bounds__(RS_T) k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                     int bits, uint32_t *__restrict__ ghist, int64_t ntiles) {
    __shared__ uint32_t h[1 << RS_MAXBITS];
    const int nb = 1 << bits;
    const uint32_t mask = nb - 1;
    for (int i = threadIdx.x; i < nb; i += RS_T) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const int lane = threadIdx.x & 31;
    uint32_t kv[RS_ITEMS];  // all loads first, so their latencies overlap
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t i = base + (int64_t)k * RS_T + threadIdx.x;
        kv[k] = i < n ? rs_key<PACKED>(keys, i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t i = base + (int64_t)k * RS_T + threadIdx.x;
        const bool valid = i < n;
        const uint32_t dg = valid ? (kv[k] >> shift) & mask : 0u;
        const unsigned peers = digit_peers(dg, bits, __ballot_sync(0xFFFFFFFFu, valid));
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[dg], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += RS_T) ghist[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

// Scatter one tile stably.  gscan = exclusive scan of ghist in digit-major order.  The first pass
// reads the cell keys (the value is the point index); later passes read the (key, index) pairs
// an earlier pass wrote.  Passes before the last write (key, index) pairs as one 8-byte store,
// the last writes the indices only (the permutation).
template <bool FIRST, bool OUT_PAIRS>
__global__ void __launch_bounds__(RS_T, 2) k_radix_scatter(const uint32_t *__restrict__ kin, uint32_t *__restrict__ out,
                                                        int64_t n, int shift, int bits,
                                                        const uint32_t *__restrict__ gscan, int64_t ntiles) {
    extern __shared__ uint32_t smem[];
    const int nb = 1 << bits;
    const uint32_t mask = nb - 1;
    uint32_t *wcnt = smem;                   // 8 x nb
    uint32_t *tstart = wcnt + 8 * nb;        // nb
    uint32_t *gbase = tstart + nb;           // nb
    uint32_t *skey = gbase + nb;             // RS_TILE
    uint32_t *sval = skey + RS_TILE;         // RS_TILE
    __shared__ uint32_t scan_sh[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // point indices fit 32 bits (the permutation is u32)
    const uint32_t base = blockIdx.x * (uint32_t)RS_TILE;
    const int tile_n = (int)min((int64_t)RS_TILE, n - (int64_t)base);
    for (int i = threadIdx.x; i < 8 * nb; i += RS_T) wcnt[i] = 0;
    __syncthreads();
    // rank of each key among the earlier keys of this warp with the same digit
    // (ranks < 1024: two 16-bit ranks per register).  The warp's 32 coalesced key loads are all
    // issued before the ranking starts, so their latencies overlap.
    // Later passes load each (key, index) pair whole (one 8-byte load) and park the index in
    // sval, in input order, until the ranks are known.
    uint32_t kr[RS_ITEMS], rk[RS_ITEMS / 2];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int s = 0; s < RS_ITEMS; ++s) {
        const int pos = w * (RS_ITEMS * 32) + s * 32 + lane;
        if (FIRST) {
            kr[s] = pos < tile_n ? __ldcs(kin + base + (uint32_t)pos) : 0u;
        } else {
            const uint2 kv = pos < tile_n ? __ldcs(reinterpret_cast<const uint2 *>(kin) + base + (uint32_t)pos)
                                          : make_uint2(0u, 0u);
            kr[s] = kv.x;
            sval[pos] = kv.y;
        }
    }
#pragma unroll
    for (int s = 0; s < RS_ITEMS; ++s) {
        const int pos = w * (RS_ITEMS * 32) + s * 32 + lane;
        const bool valid = pos < tile_n;
        const uint32_t dg = (kr[s] >> shift) & mask;
        const unsigned peers = digit_peers(dg, bits, __ballot_sync(0xFFFFFFFFu, valid));
        const uint32_t before = valid ? wcnt[w * nb + dg] : 0u;
        const uint32_t rank = before + (uint32_t)__popc(peers & lt);
        if (s & 1) rk[s >> 1] |= rank << 16; else rk[s >> 1] = rank;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[w * nb + dg] = before + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps; tile totals
    for (int dg = threadIdx.x; dg < nb; dg += RS_T) {
        uint32_t run = 0;
        for (int ww = 0; ww < 8; ++ww) {
            const uint32_t c = wcnt[ww * nb + dg];
            wcnt[ww * nb + dg] = run;
            run += c;
        }
        tstart[dg] = run;
        gbase[dg] = gscan[(int64_t)dg * ntiles + blockIdx.x];
    }
    __syncthreads();
    // exclusive scan of tile totals over digits (nb <= 1024 = 4 per thread)
    {
        uint32_t v[4];
        uint32_t sum = 0;
        for (int k = 0; k < 4; ++k) {
            const int dg = threadIdx.x * 4 + k;
            v[k] = dg < nb ? tstart[dg] : 0u;
            sum += v[k];
        }
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(sum, scan_sh, tot);
        for (int k = 0; k < 4; ++k) {
            const int dg = threadIdx.x * 4 + k;
            if (dg < nb) tstart[dg] = ex;
            ex += v[k];
        }
    }
    __syncthreads();
    uint32_t vv[FIRST ? 1 : RS_ITEMS];
    if (!FIRST) {
#pragma unroll
        for (int s = 0; s < RS_ITEMS; ++s) vv[FIRST ? 0 : s] = sval[w * (RS_ITEMS * 32) + s * 32 + lane];
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < RS_ITEMS; ++s) {
        const int pos = w * (RS_ITEMS * 32) + s * 32 + lane;
        if (pos < tile_n) {
            const uint32_t dg = (kr[s] >> shift) & mask;
            const uint32_t lp = tstart[dg] + wcnt[w * nb + dg] + ((s & 1) ? (rk[s >> 1] >> 16) : (rk[s >> 1] & 0xFFFFu));
            skey[lp] = kr[s];
            sval[lp] = FIRST ? base + (uint32_t)pos : vv[FIRST ? 0 : s];
        }
        if ((s & 7) == 7) __syncwarp();  // bounds how far the counter loads are hoisted (registers)
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tile_n; i += RS_T) {
        const uint32_t key = skey[i];
        const uint32_t dg = (key >> shift) & mask;
        const uint32_t g = gbase[dg] + ((uint32_t)i - tstart[dg]);
        const uint32_t val = sval[i];
        if (OUT_PAIRS)
            reinterpret_cast<uint2 *>(out)[g] = make_uint2(key, val);
        else
            out[g] = val;
    }
}

static size_t radix_scatter_smem(int bits) {
    const int nb = 1 << bits;
    return sizeof(uint32_t) * (size_t)(8 * nb + 2 * nb + 2 * RS_TILE);
}

// Digit width of the first pass (the others use the same width).
static int radix_pass_bits(int keybits) {
    keybits = std::max(keybits, 1);
    const int npass = (int)cdiv(keybits, RS_MAXBITS);
    return (int)cdiv(keybits, npass);
}

// Stable sort of `keys` (values < 2^keybits); writes the permutation to perm_out.  Scratch:
// pairs (2 n words per buffer; the second buffer only with three or more passes), ghist
// (2^10 * ntiles), bsum.  With first_hist, ghist already holds the first pass's per-tile
// histogram (from k_keys).
static int radix_sort_perm(const uint32_t *keys, int64_t n, int keybits, uint32_t *perm_out, uint32_t *pairs_a,
                           uint32_t *pairs_b, uint32_t *ghist, uint32_t *bsum, bool first_hist, cudaStream_t s) {
    const int64_t ntiles = cdiv(n, RS_TILE);
    keybits = std::max(keybits, 1);
    const int npass = (int)cdiv(keybits, RS_MAXBITS);
    const int bits = (int)cdiv(keybits, npass);
    {
        const size_t mx = radix_scatter_smem(RS_MAXBITS);
        FK_TRY(raise_smem_limit((const void *)k_radix_scatter<true, true>, mx));
        FK_TRY(raise_smem_limit((const void *)k_radix_scatter<true, false>, mx));
        FK_TRY(raise_smem_limit((const void *)k_radix_scatter<false, true>, mx));
        FK_TRY(raise_smem_limit((const void *)k_radix_scatter<false, false>, mx));
    }
    const uint32_t *kin = keys;
    uint32_t *pbufs[2] = {pairs_a, pairs_b};
    for (int p = 0; p < npass; ++p) {
        const int shift = p * bits;
        const int b = std::min(bits, keybits - shift);
        const bool first = p == 0, last = p == npass - 1;
        if (!(first && first_hist)) {
            if (first)
                k_radix_hist<false><<<(unsigned)ntiles, RS_T, 0, s>>>(kin, n, shift, b, ghist, ntiles);
            else
                k_radix_hist<true><<<(unsigned)ntiles, RS_T, 0, s>>>(kin, n, shift, b, ghist, ntiles);
            FK_LAUNCH();
        }
        FK_TRY(exclusive_scan_u32(ghist, ghist, ((int64_t)1 << b) * ntiles, false, bsum, s));
        uint32_t *out = last ? perm_out : pbufs[p % 2];
        const size_t sm = radix_scatter_smem(b);
        if (first && last)
            k_radix_scatter<true, false><<<(unsigned)ntiles, RS_T, sm, s>>>(kin, out, n, shift, b, ghist, ntiles);
        else if (first)
            k_radix_scatter<true, true><<<(unsigned)ntiles, RS_T, sm, s>>>(kin, out, n, shift, b, ghist, ntiles);
        else if (last)
            k_radix_scatter<false, false><<<(unsigned)ntiles, RS_T, sm, s>>>(kin, out, n, shift, b, ghist, ntiles);
        else
            k_radix_scatter<false, true><<<(unsigned)ntiles, RS_T, sm, s>>>(kin, out, n, shift, b, ghist, ntiles);
        FK_LAUNCH();
        kin = out;
    }
    return FKSKI_OK;
}

// ------------------------------------------------------------------ per-cell moments
// Tiling: a CTA owns one "column" (all cells along the last axis for fixed leading cells) and a
// range of output nodes [js, je) along the last axis; it reduces the cells [js-3, je) of that
// column (a warp per cell, in order) into shared memory, then contracts the last axis.
struct ColTiling {
    int64_t ncol;      // columns = prod_{k<d-1} (M_k - 3)
    int C;             // cells along the last axis (M_last - 3)
    int Ml;            // nodes along the last axis
    int NT;            // output nodes per tile
    int ntile;         // tiles per column
    int nct;           // cell slots per tile (shared memory)
};

template <int D>
struct MomLayout;
template <>
struct MomLayout<1> { static constexpr int NM = 7, NY = 4, SLOT = 12, PSTRIDE = 0; };
template <>
struct MomLayout<2> { static constexpr int NM = 49, NY = 16, SLOT = 68, PSTRIDE = 24; };
template <>
struct MomLayout<3> { static constexpr int NM = 343, NY = 64, SLOT = 408, PSTRIDE = 40; };

template <typename T, int D>
struct MomCap;  // cells per tile
template <> struct MomCap<float, 1> { static constexpr int NCT = 2048; };
template <> struct MomCap<double, 1> { static constexpr int NCT = 1024; };
template <> struct MomCap<float, 2> { static constexpr int NCT = 512; };
template <> struct MomCap<double, 2> { static constexpr int NCT = 256; };
template <> struct MomCap<float, 3> { static constexpr int NCT = 96; };
template <> struct MomCap<double, 3> { static constexpr int NCT = 32; };

constexpr int MOM_WARPS = 8;

// Stage 32 points of a cell segment into the warp's point buffer (Bernstein-6 and cubic weights).
template <typename T, int D>
__device__ __forceinline__ void stage_points(const uint32_t *__restrict__ perm, const Rec4<T> *__restrict__ rec,
                                             uint32_t p, uint32_t end, T *pb, int lane) {
    constexpr int PS = MomLayout<D>::PSTRIDE;
    T *q = pb + lane * PS;
    if (p < end) {
        const Rec4<T> r = rec[perm[p]];
        T b[7], w[4];
        bern6<T>(r.t[0], b);
#pragma unroll
        for (int i = 0; i < 7; ++i) q[i] = b[i];
        q[7] = r.y;
#pragma unroll
        for (int k = 1; k < D; ++k) {
            bern6<T>(r.t[k], b);
#pragma unroll
            for (int i = 0; i < 7; ++i) q[8 * k + i] = b[i];
            q[8 * k + 7] = T(0);
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            keys_weights<T>(r.t[k], w);
#pragma unroll
            for (int i = 0; i < 4; ++i) q[8 * D + 4 * k + i] = w[i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < PS; ++i) q[i] = T(0);
    }
}

// D = 3: lanes = 4 sub-groups x 8 roles; a sub-group takes every 4th point of a 32-point chunk.
// Role r < 7 accumulates M[r][p2][p3] (49); every role accumulates 8 of the 64 Y values.
template <typename T>
__device__ void cell_moments_d3(const uint32_t *__restrict__ perm, const Rec4<T> *__restrict__ rec, uint32_t beg,
                                uint32_t end, T *pb, T *slot, int lane) {
    constexpr int PS = MomLayout<3>::PSTRIDE;
    constexpr bool TWO = sizeof(T) == 4;
    const int sg = lane >> 3, r = lane & 7;
    T m1[49], y1[8];
    T m2[TWO ? 49 : 1], y2[TWO ? 8 : 1];
#pragma unroll
    for (int i = 0; i < 49; ++i) m1[i] = T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) y1[i] = T(0);
    if (TWO) {
#pragma unroll
        for (int i = 0; i < (TWO ? 49 : 1); ++i) m2[i] = T(0);
#pragma unroll
        for (int i = 0; i < (TWO ? 8 : 1); ++i) y2[i] = T(0);
    }
    int nch = 0;
    for (uint32_t c0 = beg; c0 < end; c0 += 32) {
        stage_points<T, 3>(perm, rec, c0 + lane, end, pb, lane);
        __syncwarp();
        const int npts = (int)min(32u, end - c0);
        for (int k = sg; k < npts; k += 4) {
            const T *q = pb + k * PS;
            const T alpha = r < 7 ? q[r] : T(0);
            const T yv = q[7];
            T b2[7], b3[7];
#pragma unroll
            for (int i = 0; i < 7; ++i) { b2[i] = q[8 + i]; b3[i] = q[16 + i]; }
#pragma unroll
            for (int p2 = 0; p2 < 7; ++p2) {
                const T ab = alpha * b2[p2];
#pragma unroll
                for (int p3 = 0; p3 < 7; ++p3) m1[p2 * 7 + p3] = fma(ab, b3[p3], m1[p2 * 7 + p3]);
            }
            const T ywa = yv * q[24 + (r >> 1)];
            const T q0 = ywa * q[28 + 2 * (r & 1)], q1 = ywa * q[28 + 2 * (r & 1) + 1];
#pragma unroll
            for (int a3 = 0; a3 < 4; ++a3) {
                y1[a3] = fma(q0, q[32 + a3], y1[a3]);
                y1[4 + a3] = fma(q1, q[32 + a3], y1[4 + a3]);
            }
        }
        __syncwarp();
        if (TWO && ++nch == 4) {
#pragma unroll
            for (int i = 0; i < (TWO ? 49 : 1); ++i) { m2[i] += m1[i]; m1[i] = T(0); }
#pragma unroll
            for (int i = 0; i < (TWO ? 8 : 1); ++i) { y2[i] += y1[i]; y1[i] = T(0); }
            nch = 0;
        }
    }
    if (TWO) {
#pragma unroll
        for (int i = 0; i < (TWO ? 49 : 1); ++i) m1[i] += m2[i];
#pragma unroll
        for (int i = 0; i < (TWO ? 8 : 1); ++i) y1[i] += y2[i];
    }
#pragma unroll
    for (int i = 0; i < 49; ++i) {
        m1[i] += __shfl_xor_sync(0xFFFFFFFFu, m1[i], 8);
        m1[i] += __shfl_xor_sync(0xFFFFFFFFu, m1[i], 16);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        y1[i] += __shfl_xor_sync(0xFFFFFFFFu, y1[i], 8);
        y1[i] += __shfl_xor_sync(0xFFFFFFFFu, y1[i], 16);
    }
    if (sg == 0) {
        if (r < 7) {
#pragma unroll
            for (int i = 0; i < 49; ++i) slot[r * 49 + i] = m1[i];
        }
        const int a1 = r >> 1, a2 = 2 * (r & 1);
#pragma unroll
        for (int a3 = 0; a3 < 4; ++a3) {
            slot[343 + a1 * 16 + a2 * 4 + a3] = y1[a3];
            slot[343 + a1 * 16 + (a2 + 1) * 4 + a3] = y1[4 + a3];
        }
    }
}

// D = 2: same lane roles; role r < 7 accumulates M[r][p2] (7); every role 2 of the 16 Y values.
template <typename T>
__device__ void cell_moments_d2(const uint32_t *__restrict__ perm, const Rec4<T> *__restrict__ rec, uint32_t beg,
                                uint32_t end, T *pb, T *slot, int lane) {
    constexpr int PS = MomLayout<2>::PSTRIDE;
    const int sg = lane >> 3, r = lane & 7;
    T m1[7], y1[2], m2[7], y2[2];
#pragma unroll
    for (int i = 0; i < 7; ++i) m1[i] = m2[i] = T(0);
    y1[0] = y1[1] = y2[0] = y2[1] = T(0);
    int nch = 0;
    for (uint32_t c0 = beg; c0 < end; c0 += 32) {
        stage_points<T, 2>(perm, rec, c0 + lane, end, pb, lane);
        __syncwarp();
        const int npts = (int)min(32u, end - c0);
        for (int k = sg; k < npts; k += 4) {
            const T *q = pb + k * PS;
            const T alpha = r < 7 ? q[r] : T(0);
#pragma unroll
            for (int p2 = 0; p2 < 7; ++p2) m1[p2] = fma(alpha, q[8 + p2], m1[p2]);
            const T ywa = q[7] * q[16 + (r >> 1)];
            y1[0] = fma(ywa, q[20 + 2 * (r & 1)], y1[0]);
            y1[1] = fma(ywa, q[20 + 2 * (r & 1) + 1], y1[1]);
        }
        __syncwarp();
        if (++nch == 4) {
#pragma unroll
            for (int i = 0; i < 7; ++i) { m2[i] += m1[i]; m1[i] = T(0); }
            y2[0] += y1[0]; y2[1] += y1[1]; y1[0] = y1[1] = T(0);
            nch = 0;
        }
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        T v = m1[i] + m2[i];
        v += __shfl_xor_sync(0xFFFFFFFFu, v, 8);
        v += __shfl_xor_sync(0xFFFFFFFFu, v, 16);
        m1[i] = v;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        T v = y1[i] + y2[i];
        v += __shfl_xor_sync(0xFFFFFFFFu, v, 8);
        v += __shfl_xor_sync(0xFFFFFFFFu, v, 16);
        y1[i] = v;
    }
    if (sg == 0) {
        if (r < 7) {
#pragma unroll
            for (int i = 0; i < 7; ++i) slot[r * 7 + i] = m1[i];
        }
        const int a1 = r >> 1, a2 = 2 * (r & 1);
        slot[49 + a1 * 4 + a2] = y1[0];
        slot[49 + a1 * 4 + a2 + 1] = y1[1];
    }
}

// D = 1: every lane accumulates all 11 values for its own points; warp tree at the end.
template <typename T>
__device__ void cell_moments_d1(const uint32_t *__restrict__ perm, const Rec4<T> *__restrict__ rec, uint32_t beg,
                                uint32_t end, T *slot, int lane) {
    T m1[7], y1[4], m2[7], y2[4];
#pragma unroll
    for (int i = 0; i < 7; ++i) m1[i] = m2[i] = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) y1[i] = y2[i] = T(0);
    int nch = 0;
    for (uint32_t c0 = beg; c0 < end; c0 += 32) {
        const uint32_t p = c0 + lane;
        if (p < end) {
            const Rec4<T> rr = rec[perm[p]];
            T b[7], w[4];
            bern6<T>(rr.t[0], b);
            keys_weights<T>(rr.t[0], w);
#pragma unroll
            for (int i = 0; i < 7; ++i) m1[i] += b[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) y1[i] = fma(rr.y, w[i], y1[i]);
        }
        if (++nch == 32) {
#pragma unroll
            for (int i = 0; i < 7; ++i) { m2[i] += m1[i]; m1[i] = T(0); }
#pragma unroll
            for (int i = 0; i < 4; ++i) { y2[i] += y1[i]; y1[i] = T(0); }
            nch = 0;
        }
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        T v = m1[i] + m2[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        m1[i] = v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        T v = y1[i] + y2[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        y1[i] = v;
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 7; ++i) slot[i] = m1[i];
#pragma unroll
        for (int i = 0; i < 4; ++i) slot[7 + i] = y1[i];
    }
}

// Moments of a column tile + contraction of the last axis.
// Outputs (SoA, spatial index = col * Ml + j):
//   D=3: outM[(p1*7+p2)*7 + dl][col*Ml + j], outY[(a1*4+a2)][..]
//   D=2: outM[p1*7 + dl][..], outY[a1][..]
//   D=1: outM[dl][j] (the band), outY[j] (W^T y)
template <typename T, int D>
__global__ void __launch_bounds__(MOM_WARPS * 32) k_moments(const uint32_t *__restrict__ perm, const Rec4<T> *__restrict__ rec,
                                                             const uint32_t *__restrict__ offsets, ColTiling tl,
                                                             T *__restrict__ outM, T *__restrict__ outY) {
    using L = MomLayout<D>;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *pbuf = reinterpret_cast<T *>(smraw);
    T *slots = pbuf + (L::PSTRIDE > 0 ? MOM_WARPS * 32 * L::PSTRIDE : 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t col = blockIdx.x / tl.ntile;
    const int tile = (int)(blockIdx.x % tl.ntile);
    const int js = tile * tl.NT;
    const int je = min(js + tl.NT, tl.Ml);
    const int cfirst = max(js - 3, 0);
    const int cend = min(je, tl.C);
    const int nct = cend - cfirst;
    for (int lc = warp; lc < nct; lc += MOM_WARPS) {
        const int64_t key = col * tl.C + (cfirst + lc);
        const uint32_t beg = offsets[key], end = offsets[key + 1];
        T *slot = slots + (int64_t)lc * L::SLOT;
        if (D == 3)
            cell_moments_d3<T>(perm, rec, beg, end, pbuf + warp * 32 * L::PSTRIDE, slot, lane);
        else if (D == 2)
            cell_moments_d2<T>(perm, rec, beg, end, pbuf + warp * 32 * L::PSTRIDE, slot, lane);
        else
            cell_moments_d1<T>(perm, rec, beg, end, slot, lane);
    }
    __syncthreads();
    const int nj = je - js;
    const int64_t S1 = tl.ncol * tl.Ml;
    constexpr int NCOMP = L::NM / 7;  // leading comps of M: 49 / 7 / 1
    constexpr int NYC = L::NY / 4;    // leading comps of Y: 16 / 4 / 1
    for (int it = threadIdx.x; it < NCOMP * nj; it += blockDim.x) {
        const int jj = it % nj, pp = it / nj;
        const int j = js + jj;
        T acc[7];
#pragma unroll
        for (int dl = 0; dl < 7; ++dl) acc[dl] = T(0);
        auto cell = [&](auto a_) {
            constexpr int a = decltype(a_)::value;
            const int c = j - a;
            if (c >= cfirst && c < cend) {
                const T *sl = slots + (int64_t)(c - cfirst) * L::SLOT + pp * 7;
                T v[7];
#pragma unroll
                for (int p = 0; p < 7; ++p) v[p] = sl[p];
                etab_accumulate<a>(acc, v);
            }
        };
        cell(std::integral_constant<int, 0>{});
        cell(std::integral_constant<int, 1>{});
        cell(std::integral_constant<int, 2>{});
        cell(std::integral_constant<int, 3>{});
        const int64_t sp = col * tl.Ml + j;
#pragma unroll
        for (int dl = 0; dl < 7; ++dl) outM[(int64_t)(pp * 7 + dl) * S1 + sp] = acc[dl];
    }
    for (int it = threadIdx.x; it < NYC * nj; it += blockDim.x) {
        const int jj = it % nj, yy = it / nj;
        const int j = js + jj;
        T acc = T(0);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int c = j - a;
            if (c >= cfirst && c < cend) acc += slots[(int64_t)(c - cfirst) * L::SLOT + L::NM + yy * 4 + a];
        }
        outY[(int64_t)yy * S1 + col * tl.Ml + j] = acc;
    }
}

// ------------------------------------------------------------------ FP32 3-D moments, point-balanced
// The same per-cell sums as k_moments<float, 3>, with the work of a column tile split evenly by
// points instead of by cells: warp w takes the w-th eighth of the tile's sorted point range,
// walks it cell by cell in chunks of at most 32 points of one cell, and keeps 49 + 8 FP32 sums
// per lane (4 sub-groups x 8 roles, as in cell_moments_d3).  Every M3_FLUSH chunks and at the
// end of its part of a cell it folds the sub-groups together and adds the sums to shared
// memory: straight into the cell's slot when the warp owns the whole cell, else into one of its
// two edge buffers (first / last cell, shared with the neighbouring warps).  The edge buffers
// are added to the slots in warp order afterwards, so the result does not depend on timing.
// Records of the next chunk are loaded before the current one is computed.
constexpr int M3_WARPS = 8;
constexpr int M3_PS = 36;     // staged floats per point: B1[7], y | B2[7], 0 | B3[7], 0 | w1[4] | w2[4] | w3[4]
constexpr int M3_SLOT = 409;  // 343 moments + 64 y-moments + 2 pad (odd stride: the contraction's
                              // threads read slots of consecutive cells without bank conflicts)
constexpr int M3_FLUSH = 8;   // chunks between folds of the register sums
constexpr int M3_NCT = 64;    // cells per tile

static size_t moments3f_smem(int nct) {
    return sizeof(float) * ((size_t)M3_WARPS * 32 * M3_PS + (size_t)nct * M3_SLOT + (size_t)M3_WARPS * 2 * M3_SLOT) +
           sizeof(uint32_t) * (size_t)(nct + 1) + sizeof(int) * 2 * M3_WARPS;
}

__device__ __forceinline__ int m3_find_cell(const uint32_t *coff, int nct, uint32_t p) {
    int lo = 0, hi = nct - 1;  // largest i with coff[i] <= p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (coff[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(M3_WARPS * 32) k_moments3f(const uint32_t *__restrict__ perm, const Rec4<float> *__restrict__ rec,
                                                              const uint32_t *__restrict__ offsets, ColTiling tl,
                                                              float *__restrict__ outM, float *__restrict__ outY) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sg = lane >> 3, r = lane & 7;
    const int64_t col = blockIdx.x / tl.ntile;
    const int tile = (int)(blockIdx.x % tl.ntile);
    const int js = tile * tl.NT;
    const int je = min(js + tl.NT, tl.Ml);
    const int cfirst = max(js - 3, 0);
    const int cend = min(je, tl.C);
    const int nct = cend - cfirst;
    float *stage = reinterpret_cast<float *>(smraw);
    float *slots = stage + M3_WARPS * 32 * M3_PS;
    float *edge = slots + nct * M3_SLOT;
    uint32_t *coff = reinterpret_cast<uint32_t *>(edge + M3_WARPS * 2 * M3_SLOT);
    int *ecell = reinterpret_cast<int *>(coff + nct + 1);
    const int64_t key0 = col * tl.C + cfirst;
    for (int i = threadIdx.x; i <= nct; i += blockDim.x) coff[i] = offsets[key0 + i];
    for (int i = threadIdx.x; i < nct * M3_SLOT + M3_WARPS * 2 * M3_SLOT; i += blockDim.x) slots[i] = 0.f;
    __syncthreads();
    const uint32_t P0 = coff[0], len = coff[nct] - P0;
    const uint32_t ws = P0 + (uint32_t)(((uint64_t)len * warp) / M3_WARPS);
    const uint32_t we = P0 + (uint32_t)(((uint64_t)len * (warp + 1)) / M3_WARPS);
    int e0 = -1, e1 = -1;
    if (ws < we) {
        const int cw = m3_find_cell(coff, nct, ws);
        const int cl = m3_find_cell(coff, nct, we - 1);
        if (coff[cw] < ws || coff[cw + 1] > we) e0 = cw;
        if (cl != cw && coff[cl + 1] > we) e1 = cl;
    }
    if (lane == 0) {
        ecell[2 * warp] = e0;
        ecell[2 * warp + 1] = e1;
    }
    float *pb = stage + warp * 32 * M3_PS;
    // moment sums of this lane's row a = r: (b, c) for b in pairs {0,1}, {2,3}, {4,5} as packed
    // float2 (updated with the paired fma.rn.f32x2, each component rounded exactly as a scalar
    // fmaf), b = 6 scalar; y sums in pairs
    float2 mp[3][7];
    float m6[7];
    float2 yp[4];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        mp[0][c] = mp[1][c] = mp[2][c] = make_float2(0.f, 0.f);
        m6[c] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) yp[i] = make_float2(0.f, 0.f);
    // component (b, c) of the lane's sums
    auto mref = [&](int b, int c) -> float & { return b == 6 ? m6[c] : ((b & 1) ? mp[b >> 1][c].y : mp[b >> 1][c].x); };
    auto yref = [&](int i) -> float & { return (i & 1) ? yp[i >> 1].y : yp[i >> 1].x; };
    uint32_t p = ws;
    int c = ws < we ? m3_find_cell(coff, nct, ws) : 0;
    int nh = ws < we ? (int)min(32u, min(coff[c + 1], we) - p) : 0;
    Rec4<float> my;
    my.t[0] = my.t[1] = my.t[2] = my.y = 0.f;
    if (lane < nh) my = rec[perm[p + lane]];
    int nacc = 0;
    while (p < we) {
        // stage this chunk (one point per lane)
        if (lane < nh) {
            float b[7], w[4], q[M3_PS];
            bern6<float>(my.t[0], b);
#pragma unroll
            for (int i = 0; i < 7; ++i) q[i] = b[i];
            q[7] = my.y;
            bern6<float>(my.t[1], b);
#pragma unroll
            for (int i = 0; i < 7; ++i) q[8 + i] = b[i];
            q[15] = 0.f;
            bern6<float>(my.t[2], b);
#pragma unroll
            for (int i = 0; i < 7; ++i) q[16 + i] = b[i];
            q[23] = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                keys_weights<float>(my.t[k], w);
#pragma unroll
                for (int i = 0; i < 4; ++i) q[24 + 4 * k + i] = w[i];
            }
            float4 *dst = reinterpret_cast<float4 *>(pb + lane * M3_PS);
#pragma unroll
            for (int v = 0; v < M3_PS / 4; ++v) dst[v] = make_float4(q[4 * v], q[4 * v + 1], q[4 * v + 2], q[4 * v + 3]);
        }
        // next chunk: skip to the cell holding p + nh, prefetch its records
        const uint32_t pn = p + (uint32_t)nh;
        const bool cell_done = pn == coff[c + 1] || pn >= we;
        int cn = c;
        int nhn = 0;
        if (pn < we) {
            while (coff[cn + 1] <= pn) ++cn;
            nhn = (int)min(32u, min(coff[cn + 1], we) - pn);
            if (lane < nhn) my = rec[perm[pn + lane]];
        }
        __syncwarp();
#pragma unroll 2
        for (int k = sg; k < nh; k += 4) {
            const float *q = pb + k * M3_PS;
            const float alpha = r < 7 ? q[r] : 0.f;
            const float yv = q[7];
            const float4 b2a = *reinterpret_cast<const float4 *>(q + 8), b2b = *reinterpret_cast<const float4 *>(q + 12);
            const float4 b3a = *reinterpret_cast<const float4 *>(q + 16), b3b = *reinterpret_cast<const float4 *>(q + 20);
            const float b3[7] = {b3a.x, b3a.y, b3a.z, b3a.w, b3b.x, b3b.y, b3b.z};
            // ab_b = alpha * B2_b (rounded), then sum_c += ab_b * B3_c
            const float2 aa = make_float2(alpha, alpha);
            const float2 ab01 = __fmul2_rn(aa, make_float2(b2a.x, b2a.y));
            const float2 ab23 = __fmul2_rn(aa, make_float2(b2a.z, b2a.w));
            const float2 ab45 = __fmul2_rn(aa, make_float2(b2b.x, b2b.y));
            const float ab6 = alpha * b2b.z;
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                const float2 zz = make_float2(b3[c], b3[c]);
                mp[0][c] = __ffma2_rn(ab01, zz, mp[0][c]);
                mp[1][c] = __ffma2_rn(ab23, zz, mp[1][c]);
                mp[2][c] = __ffma2_rn(ab45, zz, mp[2][c]);
                m6[c] = fmaf(ab6, b3[c], m6[c]);
            }
            const float ywa = yv * q[24 + (r >> 1)];
            const float2 w2 = *reinterpret_cast<const float2 *>(q + 28 + 2 * (r & 1));
            const float4 w3 = *reinterpret_cast<const float4 *>(q + 32);
            const float2 qq = __fmul2_rn(make_float2(ywa, ywa), w2);
            const float2 q0 = make_float2(qq.x, qq.x), q1 = make_float2(qq.y, qq.y);
            const float2 w3a = make_float2(w3.x, w3.y), w3b = make_float2(w3.z, w3.w);
            yp[0] = __ffma2_rn(q0, w3a, yp[0]);
            yp[1] = __ffma2_rn(q0, w3b, yp[1]);
            yp[2] = __ffma2_rn(q1, w3a, yp[2]);
            yp[3] = __ffma2_rn(q1, w3b, yp[3]);
        }
        __syncwarp();
        if (cell_done || ++nacc == M3_FLUSH) {
#pragma unroll
            for (int b = 0; b < 7; ++b)
#pragma unroll
                for (int c = 0; c < 7; ++c) {
                    float &v = mref(b, c);
                    v += __shfl_xor_sync(0xFFFFFFFFu, v, 8);
                    v += __shfl_xor_sync(0xFFFFFFFFu, v, 16);
                }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float &v = yref(i);
                v += __shfl_xor_sync(0xFFFFFFFFu, v, 8);
                v += __shfl_xor_sync(0xFFFFFFFFu, v, 16);
            }
            if (sg == 0) {
                float *dst = c == e0 ? edge + (warp * 2) * M3_SLOT
                                     : (c == e1 ? edge + (warp * 2 + 1) * M3_SLOT : slots + c * M3_SLOT);
                if (r < 7) {
#pragma unroll
                    for (int b = 0; b < 7; ++b)
#pragma unroll
                        for (int c = 0; c < 7; ++c) dst[r * 49 + b * 7 + c] += mref(b, c);
                }
                const int a1 = r >> 1, a2 = 2 * (r & 1);
#pragma unroll
                for (int a3 = 0; a3 < 4; ++a3) {
                    dst[343 + a1 * 16 + a2 * 4 + a3] += yref(a3);
                    dst[343 + a1 * 16 + (a2 + 1) * 4 + a3] += yref(4 + a3);
                }
            }
            __syncwarp();
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                mp[0][c] = mp[1][c] = mp[2][c] = make_float2(0.f, 0.f);
                m6[c] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) yp[i] = make_float2(0.f, 0.f);
            nacc = 0;
        }
        p = pn;
        c = cn;
        nh = nhn;
    }
    __syncthreads();
    // edge partials into their cells, in warp order
    for (int i = threadIdx.x; i < M3_SLOT; i += blockDim.x) {
        for (int w = 0; w < M3_WARPS; ++w) {
            const int a = ecell[2 * w], b = ecell[2 * w + 1];
            if (a >= 0) slots[a * M3_SLOT + i] += edge[(w * 2) * M3_SLOT + i];
            if (b >= 0) slots[b * M3_SLOT + i] += edge[(w * 2 + 1) * M3_SLOT + i];
        }
    }
    __syncthreads();
    // last-axis contraction (as in k_moments)
    const int nj = je - js;
    const int64_t S1 = tl.ncol * tl.Ml;
    for (int it = threadIdx.x; it < 49 * nj; it += blockDim.x) {
        const int jj = it % nj, pp = it / nj;
        const int j = js + jj;
        float acc[7];
#pragma unroll
        for (int dl = 0; dl < 7; ++dl) acc[dl] = 0.f;
        auto cell = [&](auto a_) {
            constexpr int a = decltype(a_)::value;
            const int cc = j - a;
            if (cc >= cfirst && cc < cend) {
                const float *sl = slots + (cc - cfirst) * M3_SLOT + pp * 7;
                float v[7];
#pragma unroll
                for (int q = 0; q < 7; ++q) v[q] = sl[q];
                etab_accumulate<a>(acc, v);
            }
        };
        cell(std::integral_constant<int, 0>{});
        cell(std::integral_constant<int, 1>{});
        cell(std::integral_constant<int, 2>{});
        cell(std::integral_constant<int, 3>{});
        const int64_t sp = col * tl.Ml + j;
#pragma unroll
        for (int dl = 0; dl < 7; ++dl) outM[(int64_t)(pp * 7 + dl) * S1 + sp] = acc[dl];
    }
    for (int it = threadIdx.x; it < 16 * nj; it += blockDim.x) {
        const int jj = it % nj, yy = it / nj;
        const int j = js + jj;
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int cc = j - a;
            if (cc >= cfirst && cc < cend) acc += slots[(cc - cfirst) * M3_SLOT + 343 + yy * 4 + a];
        }
        outY[(int64_t)yy * S1 + col * tl.Ml + j] = acc;
    }
}

// ------------------------------------------------------------------ probe moments
// For a group of up to 16 probes: per cell Yz[t][a] = sum_i z_t(i) prod_k w_{a_k}(t_ik).
// Lane = (h, t): t = lane & 15 (probe in group), h = lane >> 4 picks a1 in {2h, 2h+1}.
constexpr int PG = 16;

template <int D>
struct ProbeLayout;
template <> struct ProbeLayout<1> { static constexpr int NA = 4, ACC = 2, SLOT = PG * 4; };
template <> struct ProbeLayout<2> { static constexpr int NA = 16, ACC = 8, SLOT = PG * 16; };
template <> struct ProbeLayout<3> { static constexpr int NA = 64, ACC = 32, SLOT = PG * 64; };

template <typename T, int D>
struct ProbeCap;
template <> struct ProbeCap<float, 1> { static constexpr int NCT = 512; };
template <> struct ProbeCap<double, 1> { static constexpr int NCT = 256; };
template <> struct ProbeCap<float, 2> { static constexpr int NCT = 160; };
template <> struct ProbeCap<double, 2> { static constexpr int NCT = 80; };
template <> struct ProbeCap<float, 3> { static constexpr int NCT = 40; };
template <> struct ProbeCap<double, 3> { static constexpr int NCT = 20; };

template <typename T, int D>
__global__ void __launch_bounds__(MOM_WARPS * 32) k_probe_moments(const uint32_t *__restrict__ perm, const Rec4<T> *__restrict__ rec,
                                                                   const uint32_t *__restrict__ offsets, ColTiling tl,
                                                                   const T *__restrict__ Z, int64_t n, int nprobe, int t0,
                                                                   uint64_t seed, T *__restrict__ outZ) {
    using L = ProbeLayout<D>;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *pbuf = reinterpret_cast<T *>(smraw);              // MOM_WARPS x 32 x 16
    T *slots = pbuf + MOM_WARPS * 32 * 16;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tp = lane & 15, h = lane >> 4;
    const int t = t0 + tp;
    const bool active = t < nprobe;
    const int64_t col = blockIdx.x / tl.ntile;
    const int tile = (int)(blockIdx.x % tl.ntile);
    const int js = tile * tl.NT;
    const int je = min(js + tl.NT, tl.Ml);
    const int cfirst = max(js - 3, 0);
    const int cend = min(je, tl.C);
    const int nct = cend - cfirst;
    T *pb = pbuf + warp * 32 * 16;
    for (int lc = warp; lc < nct; lc += MOM_WARPS) {
        const int64_t key = col * tl.C + (cfirst + lc);
        const uint32_t beg = offsets[key], end = offsets[key + 1];
        T acc[L::ACC], acc2[L::ACC];
#pragma unroll
        for (int i = 0; i < L::ACC; ++i) acc[i] = acc2[i] = T(0);
        int nch = 0;
        for (uint32_t c0 = beg; c0 < end; c0 += 32) {
            const uint32_t p = c0 + lane;
            T *q = pb + lane * 16;
            if (p < end) {
                const uint32_t idx = perm[p];
                const Rec4<T> r = rec[idx];
                T w[4];
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    keys_weights<T>(r.t[k], w);
#pragma unroll
                    for (int i = 0; i < 4; ++i) q[4 * k + i] = w[i];
                }
                *reinterpret_cast<uint32_t *>(q + 12) = idx;
            }
            __syncwarp();
            const int npts = (int)min(32u, end - c0);
            for (int k = 0; k < npts; ++k) {
                const T *qq = pb + k * 16;
                const uint32_t idx = *reinterpret_cast<const uint32_t *>(qq + 12);
                T z = T(0);
                if (active) z = Z ? Z[(int64_t)t * n + idx] : rademacher<T>(seed, t, (int64_t)idx);
                if (D == 1) {
                    acc[0] = fma(z, qq[2 * h], acc[0]);
                    acc[1] = fma(z, qq[2 * h + 1], acc[1]);
                } else if (D == 2) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const T zw = z * qq[2 * h + e];
#pragma unroll
                        for (int a2 = 0; a2 < 4; ++a2) acc[e * 4 + a2] = fma(zw, qq[4 + a2], acc[e * 4 + a2]);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const T zw = z * qq[2 * h + e];
#pragma unroll
                        for (int a2 = 0; a2 < 4; ++a2) {
                            const T zww = zw * qq[4 + a2];
#pragma unroll
                            for (int a3 = 0; a3 < 4; ++a3)
                                acc[(e * 4 + a2) * 4 + a3] = fma(zww, qq[8 + a3], acc[(e * 4 + a2) * 4 + a3]);
                        }
                    }
                }
            }
            __syncwarp();
            if (++nch == 4) {
#pragma unroll
                for (int i = 0; i < L::ACC; ++i) { acc2[i] += acc[i]; acc[i] = T(0); }
                nch = 0;
            }
        }
        T *slot = slots + (int64_t)lc * L::SLOT + tp * L::NA + h * (L::NA / 2);
#pragma unroll
        for (int i = 0; i < L::ACC; ++i) slot[i] = acc[i] + acc2[i];
    }
    __syncthreads();
    // last-axis contraction: outZ[(t, a_1..a_{d-1})][col*Ml + j]
    const int nj = je - js;
    const int64_t S1 = tl.ncol * tl.Ml;
    constexpr int NL = L::NA / 4;  // leading components per probe
    const int ng = min(PG, nprobe - t0);
    for (int it = threadIdx.x; it < ng * NL * nj; it += blockDim.x) {
        const int jj = it % nj, rest = it / nj;
        const int lead = rest % NL, tt = rest / NL;
        const int j = js + jj;
        T a = T(0);
#pragma unroll
        for (int aa = 0; aa < 4; ++aa) {
            const int c = j - aa;
            if (c >= cfirst && c < cend) a += slots[(int64_t)(c - cfirst) * L::SLOT + tt * L::NA + lead * 4 + aa];
        }
        outZ[(int64_t)((t0 + tt) * NL + lead) * S1 + col * tl.Ml + j] = a;
    }
}

// ------------------------------------------------------------------ generic axis contraction
// in : comps (co, p in [0,P), ci) x spatial (so, s in [0,S_in), si)
// out: comps (co, dl in [0,DO), ci) x spatial (so, j in [0,S_out), si)
// out = sum_{a = 0..3, 0 <= j-a < S_in} sum_p E[a][dl][p] in[p][j-a]     (M part, P = DO = 7)
// out = sum_{a = 0..3, 0 <= j-a < S_in} in[a][j-a]                       (Y part, P = 4, DO = 1)
struct AxisPass {
    int64_t n_co, n_ci, n_so, n_si;
    int S_in, S_out;
};

// One thread owns a run of AXJ consecutive output nodes j along the contracted axis (fixed
// co, ci, so, si) and slides over the cells j-3 .. j+AXJ-1 once: each cell's values are loaded
// once per run instead of once per output (4x fewer loads).  Consecutive threads take
// consecutive si, so loads and stores stay coalesced.
constexpr int AXJ = 8;

template <typename T, bool MPART>
__global__ void __launch_bounds__(256) k_axis_pass(const T *__restrict__ in, T *__restrict__ out, AxisPass ap) {
    constexpr int P = MPART ? 7 : 4;
    constexpr int DO = MPART ? 7 : 1;
    const int64_t Sin_tot = ap.n_so * ap.S_in * ap.n_si;
    const int64_t Sout_tot = ap.n_so * ap.S_out * ap.n_si;
    const int nrun = (ap.S_out + AXJ - 1) / AXJ;
    const int64_t total = ap.n_co * ap.n_ci * ap.n_so * nrun * ap.n_si;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = it;
        const int64_t si = r % ap.n_si; r /= ap.n_si;
        const int jr = (int)(r % nrun); r /= nrun;
        const int64_t so = r % ap.n_so; r /= ap.n_so;
        const int64_t ci = r % ap.n_ci;
        const int64_t co = r / ap.n_ci;
        const int j0 = jr * AXJ;
        const int jn = min(AXJ, ap.S_out - j0);
        // component p of cell c at src[p * pstr + c * n_si]; output dl of node j at dst[dl * dstr + j * n_si]
        const int64_t pstr = ap.n_ci * Sin_tot, dstr = ap.n_ci * Sout_tot;
        const T *src = in + (co * P * ap.n_ci + ci) * Sin_tot + so * ap.S_in * ap.n_si + si;
        T *dst = out + (co * DO * ap.n_ci + ci) * Sout_tot + so * ap.S_out * ap.n_si + si;
        // win[3 - a] holds cell j - a; the window shifts by one cell per output
        T win[4][P];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int c = j0 - 3 + k;
            const T *q = src + (int64_t)c * ap.n_si;
#pragma unroll
            for (int p = 0; p < P; ++p) win[k + 1][p] = (c >= 0 && c < ap.S_in) ? q[p * pstr] : T(0);
        }
#pragma unroll 1
        for (int jj = 0; jj < jn; ++jj) {
            const int j = j0 + jj;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int p = 0; p < P; ++p) win[k][p] = win[k + 1][p];
            const T *q = src + (int64_t)j * ap.n_si;
#pragma unroll
            for (int p = 0; p < P; ++p) win[3][p] = (j < ap.S_in) ? q[p * pstr] : T(0);
            T acc[DO];
#pragma unroll
            for (int dl = 0; dl < DO; ++dl) acc[dl] = T(0);
            if constexpr (MPART) {
                // cell j - a is win[3 - a]
                etab_accumulate<0>(acc, win[3]);
                etab_accumulate<1>(acc, win[2]);
                etab_accumulate<2>(acc, win[1]);
                etab_accumulate<3>(acc, win[0]);
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a) acc[0] += win[3 - a][a];
            }
            T *o = dst + (int64_t)j * ap.n_si;
#pragma unroll
            for (int dl = 0; dl < DO; ++dl) o[dl * dstr] = acc[dl];
        }
    }
}

template <typename T, bool MPART>
static int launch_axis_pass(const T *in, T *out, AxisPass ap, cudaStream_t s) {
    const int64_t total = ap.n_co * ap.n_ci * ap.n_so * ((ap.S_out + AXJ - 1) / AXJ) * ap.n_si;
    const int64_t nb = std::min<int64_t>(cdiv(total, 256), 152 * 16);
    k_axis_pass<T, MPART><<<(unsigned)std::max<int64_t>(nb, 1), 256, 0, s>>>(in, out, ap);
    FK_LAUNCH();
    return FKSKI_OK;
}

// ------------------------------------------------------------------ device memory helper
struct Scratch {
    std::vector<void *> ptrs;
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <typename P>
    int get(P **p, size_t bytes) {
        void *q = nullptr;
        FK_TRY(pool_alloc(&q, bytes, s));
        ptrs.push_back(q);
        *p = reinterpret_cast<P *>(q);
        return FKSKI_OK;
    }
    ~Scratch() {
        for (void *q : ptrs) cudaFreeAsync(q, s);
    }
};

// One tile per column when the column's cells fit the shared-memory capacity; otherwise tiles
// of cap-3 output nodes, each reducing its cells [js-3, je) (the 3-cell halo is recomputed).
template <typename T, int D>
static int make_tiling(const fkski_grid &g, int nct_cap, ColTiling &tl) {
    tl.ncol = 1;
    for (int k = 0; k < D - 1; ++k) tl.ncol *= g.M[k] - 3;
    tl.Ml = (int)g.M[D - 1];
    tl.C = tl.Ml - 3;
    if (tl.C <= nct_cap) {
        tl.NT = tl.Ml;
        tl.ntile = 1;
        tl.nct = tl.C;
    } else {
        tl.NT = nct_cap - 3;
        tl.ntile = (int)cdiv(tl.Ml, tl.NT);
        tl.nct = nct_cap;
    }
    return FKSKI_OK;
}

// Band / W^T y / W^T z from the per-cell reduction.
template <typename T, int D>
static int reduce_and_assemble(fkski_stats *st, const uint32_t *perm, const Rec4<T> *rec, const uint32_t *offsets,
                               const T *Z, Scratch &sc, cudaStream_t s) {
    const fkski_grid &g = st->grid;
    using L = MomLayout<D>;
    ColTiling tl;
    make_tiling<T, D>(g, MomCap<T, D>::NCT, tl);
    const int64_t S1 = tl.ncol * tl.Ml;
    T *band = reinterpret_cast<T *>(st->band);
    T *wty = reinterpret_cast<T *>(st->wty);
    // intermediates
    T *t1 = nullptr, *t1y = nullptr, *t2 = nullptr, *t2y = nullptr;
    if (D == 1) {
        t1 = band;
        t1y = wty;
    } else {
        FK_TRY(sc.get(&t1, sizeof(T) * (size_t)(L::NM * S1)));
        FK_TRY(sc.get(&t1y, sizeof(T) * (size_t)((L::NY / 4) * S1)));
    }
    if constexpr (std::is_same<T, float>::value && D == 3) {
        ColTiling t3;
        make_tiling<T, D>(g, M3_NCT, t3);
        const size_t smem = moments3f_smem(t3.nct);
        FK_TRY(raise_smem_limit((const void *)k_moments3f, smem));
        k_moments3f<<<(unsigned)(t3.ncol * t3.ntile), M3_WARPS * 32, smem, s>>>(perm, rec, offsets, t3, t1, t1y);
    } else {
        const size_t smem = sizeof(T) * ((size_t)(L::PSTRIDE > 0 ? MOM_WARPS * 32 * L::PSTRIDE : 0) +
                                         (size_t)tl.nct * L::SLOT);
        FK_TRY(raise_smem_limit((const void *)k_moments<T, D>, smem));
        k_moments<T, D><<<(unsigned)(tl.ncol * tl.ntile), MOM_WARPS * 32, smem, s>>>(perm, rec, offsets, tl, t1, t1y);
    }
    FK_LAUNCH();
    const int64_t M0 = g.M[0];
    if (D == 3) {
        const int64_t M1 = g.M[1], M2 = g.M[2];
        FK_TRY(sc.get(&t2, sizeof(T) * (size_t)(343 * (M0 - 3) * M1 * M2)));
        FK_TRY(sc.get(&t2y, sizeof(T) * (size_t)(4 * (M0 - 3) * M1 * M2)));
        AxisPass a1{7, 7, M0 - 3, M2, (int)(M1 - 3), (int)M1};
        FK_TRY((launch_axis_pass<T, true>(t1, t2, a1, s)));
        AxisPass a0{1, 49, 1, M1 * M2, (int)(M0 - 3), (int)M0};
        FK_TRY((launch_axis_pass<T, true>(t2, band, a0, s)));
        AxisPass y1{4, 1, M0 - 3, M2, (int)(M1 - 3), (int)M1};
        FK_TRY((launch_axis_pass<T, false>(t1y, t2y, y1, s)));
        AxisPass y0{1, 1, 1, M1 * M2, (int)(M0 - 3), (int)M0};
        FK_TRY((launch_axis_pass<T, false>(t2y, wty, y0, s)));
    } else if (D == 2) {
        const int64_t M1 = g.M[1];
        AxisPass a0{1, 7, 1, M1, (int)(M0 - 3), (int)M0};
        FK_TRY((launch_axis_pass<T, true>(t1, band, a0, s)));
        AxisPass y0{1, 1, 1, M1, (int)(M0 - 3), (int)M0};
        FK_TRY((launch_axis_pass<T, false>(t1y, wty, y0, s)));
    }
    // probes
    if (st->nprobes > 0) {
        using PL = ProbeLayout<D>;
        ColTiling tp;
        make_tiling<T, D>(g, ProbeCap<T, D>::NCT, tp);
        const int64_t SP = tp.ncol * tp.Ml;
        T *wtz = reinterpret_cast<T *>(st->wtz);
        T *z1 = nullptr, *z2 = nullptr;
        constexpr int NL = PL::NA / 4;
        if (D == 1) {
            z1 = wtz;
        } else {
            FK_TRY(sc.get(&z1, sizeof(T) * (size_t)(st->nprobes * NL * SP)));
        }
        const size_t psm = sizeof(T) * ((size_t)MOM_WARPS * 32 * 16 + (size_t)tp.nct * PL::SLOT);
        FK_TRY(raise_smem_limit((const void *)k_probe_moments<T, D>, psm));
        for (int t0 = 0; t0 < st->nprobes; t0 += PG) {
            k_probe_moments<T, D><<<(unsigned)(tp.ncol * tp.ntile), MOM_WARPS * 32, psm, s>>>(
                perm, rec, offsets, tp, Z, st->n, st->nprobes, t0, st->probe_seed, z1);
            FK_LAUNCH();
        }
        if (D == 3) {
            const int64_t M1 = g.M[1], M2 = g.M[2];
            FK_TRY(sc.get(&z2, sizeof(T) * (size_t)(st->nprobes * 4 * (M0 - 3) * M1 * M2)));
            AxisPass p1{(int64_t)st->nprobes * 4, 1, M0 - 3, M2, (int)(M1 - 3), (int)M1};
            FK_TRY((launch_axis_pass<T, false>(z1, z2, p1, s)));
            AxisPass p0{(int64_t)st->nprobes, 1, 1, M1 * M2, (int)(M0 - 3), (int)M0};
            FK_TRY((launch_axis_pass<T, false>(z2, wtz, p0, s)));
        } else if (D == 2) {
            const int64_t M1 = g.M[1];
            AxisPass p0{(int64_t)st->nprobes, 1, 1, M1, (int)(M0 - 3), (int)M0};
            FK_TRY((launch_axis_pass<T, false>(z1, wtz, p0, s)));
        }
    }
    return FKSKI_OK;
}

template <typename T, int D>
static int precompute_typed(fkski_stats *st, const T *X, const T *y, const T *Z, const fkski_opts *opts,
                            cudaStream_t s) {
    Scratch sc(s);
    const int64_t n = st->n;
    const KeyParams kp = make_key_params(st->grid);
    uint32_t *keys, *counts, *offsets, *perm, *pairs_a, *pairs_b = nullptr, *ghist, *bsum;
    Rec4<T> *rec;
    int *dstatus;
    double *ypart, *dyty;
    const int64_t ncell = st->ncells;
    const int64_t ntiles = cdiv(n, RS_TILE);
    const int64_t maxscan = std::max<int64_t>(((int64_t)1 << RS_MAXBITS) * ntiles, ncell + 1);
    FK_TRY(sc.get(&keys, sizeof(uint32_t) * n));
    FK_TRY(sc.get(&rec, sizeof(Rec4<T>) * n));
    FK_TRY(sc.get(&counts, sizeof(uint32_t) * (ncell + 1)));
    FK_TRY(sc.get(&offsets, sizeof(uint32_t) * (ncell + 1)));
    FK_TRY(sc.get(&perm, sizeof(uint32_t) * n));
    int keybits = 1;
    while (((int64_t)1 << keybits) < ncell) ++keybits;
    FK_TRY(sc.get(&pairs_a, sizeof(uint2) * n));
    if (cdiv(keybits, RS_MAXBITS) > 2) FK_TRY(sc.get(&pairs_b, sizeof(uint2) * n));
    FK_TRY(sc.get(&ghist, sizeof(uint32_t) * ((int64_t)1 << RS_MAXBITS) * ntiles));
    FK_TRY(sc.get(&bsum, sizeof(uint32_t) * (cdiv(maxscan, SCAN_TILE) + 1)));
    FK_TRY(sc.get(&dstatus, sizeof(int) * 4));
    const int kblocks = (int)std::min<int64_t>(ntiles, 152 * 8);
    FK_TRY(sc.get(&ypart, sizeof(double) * (kblocks + 64 * 1216)));
    FK_TRY(sc.get(&dyty, sizeof(double) * (1 + kMaxProbes)));
    FK_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (ncell + 1), s));
    FK_CUDA(cudaMemsetAsync(dstatus, 0, sizeof(int) * 4, s));
    k_keys<T, D><<<kblocks, RS_T, 0, s>>>(X, y, n, kp, keys, rec, counts, ypart, dstatus, ghist,
                                         radix_pass_bits(keybits), ntiles);
    FK_LAUNCH();
    k_sum_partials<<<1, 32, 0, s>>>(ypart, kblocks, 1, dyty);
    FK_LAUNCH();
    FK_TRY(exclusive_scan_u32(counts, offsets, ncell, true, bsum, s));
    FK_TRY(radix_sort_perm(keys, n, keybits, perm, pairs_a, pairs_b, ghist, bsum, true, s));
    FK_TRY((reduce_and_assemble<T, D>(st, perm, rec, offsets, Z, sc, s)));
    if (st->nprobes > 0) {
        if (Z) {
            const int zb = 1216;
            k_rowsq_partials<T><<<zb, 256, 0, s>>>(Z, n, st->nprobes, ypart + kblocks, dstatus);
            FK_LAUNCH();
            k_sum_partials<<<1, 64, 0, s>>>(ypart + kblocks, zb, st->nprobes, dyty + 1);
            FK_LAUNCH();
        }
    }
    if (opts && opts->keep_sort) {
        FK_CUDA(cudaMallocAsync((void **)&st->keys, sizeof(uint32_t) * n, s));
        FK_CUDA(cudaMallocAsync((void **)&st->perm, sizeof(uint32_t) * n, s));
        FK_CUDA(cudaMemcpyAsync(st->keys, keys, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
        FK_CUDA(cudaMemcpyAsync(st->perm, perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    if (opts && (opts->keep_sort || opts->keep_points)) {
        FK_CUDA(cudaMallocAsync((void **)&st->offsets, sizeof(uint32_t) * (ncell + 1), s));
        FK_CUDA(cudaMemcpyAsync(st->offsets, offsets, sizeof(uint32_t) * (ncell + 1), cudaMemcpyDeviceToDevice, s));
    }
    if (opts && opts->keep_points) {
        FK_CUDA(cudaMallocAsync((void **)&st->pts, sizeof(Rec4<T>) * n, s));
        FK_CUDA(cudaMallocAsync((void **)&st->pkeys, sizeof(uint32_t) * n, s));
        const unsigned gbk = (unsigned)std::min<int64_t>(cdiv(n, 256), 152 * 16);
        k_gather_points<T><<<gbk, 256, 0, s>>>(perm, keys, rec, n, (Rec4<T> *)st->pts, st->pkeys);
        FK_LAUNCH();
    }
    int hstatus[4] = {0, 0, 0, 0};
    double hy[1 + kMaxProbes];
    FK_CUDA(cudaMemcpyAsync(hstatus, dstatus, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaMemcpyAsync(hy, dyty, sizeof(double) * (1 + kMaxProbes), cudaMemcpyDeviceToHost, s));
    FK_CUDA(cudaStreamSynchronize(s));
    st->yty = hy[0];
    for (int p = 0; p < st->nprobes; ++p) st->ztz[p] = Z ? hy[1 + p] : (double)n;
    return status_from_bits(hstatus[0]);
}

void destroy_stats(fkski_stats *st);

// Device address of an input array: device (or managed) memory as is; page-locked host memory
// through its device mapping; anything else (pageable host memory) is rejected.
static int device_view(const void *p, const void **dp) {
    *dp = nullptr;
    if (!p) return FKSKI_OK;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return FKSKI_E_INVALID_ARG;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        *dp = p;
        return FKSKI_OK;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *dp = a.devicePointer;
        return FKSKI_OK;
    }
    return FKSKI_E_INVALID_ARG;
}

int precompute_impl(const fkski_grid *grid, const void *X, const void *y, const void *Z, int64_t n, int dtype,
                    const fkski_opts *opts, fkski_stats **out, cudaStream_t s) {
    if (!out) return FKSKI_E_INVALID_ARG;
    *out = nullptr;
    if (!grid || !X || !y || n < 1) return FKSKI_E_INVALID_ARG;
    if (dtype != FKSKI_F32 && dtype != FKSKI_F64) return FKSKI_E_INVALID_ARG;
    FK_TRY(device_view(X, &X));
    FK_TRY(device_view(y, &y));
    FK_TRY(device_view(Z, &Z));
    const int d = grid->d;
    if (d < 1 || d > 3) return FKSKI_E_INVALID_ARG;
    int64_t m = 1, ncell = 1;
    for (int k = 0; k < d; ++k) {
        if (grid->M[k] < 4 || !(grid->h[k] > 0.0) || !std::isfinite(grid->h[k]) || !std::isfinite(grid->lo[k]))
            return FKSKI_E_INVALID_ARG;
        if (grid->M[k] > (1 << 22)) return FKSKI_E_UNSUPPORTED;
        m *= grid->M[k];
        ncell *= grid->M[k] - 3;
    }
    const int np = opts ? opts->n_probes : 0;
    if (np < 0) return FKSKI_E_INVALID_ARG;
    if (np > kMaxProbes) return FKSKI_E_UNSUPPORTED;
    if (n >= ((int64_t)1 << 31) || ncell >= ((int64_t)1 << 31) || m >= ((int64_t)1 << 31)) return FKSKI_E_UNSUPPORTED;
    // tiling capacity along the last axis is handled by tiles; nothing else to check
    fkski_stats *st = new fkski_stats;
    memset(st, 0, sizeof(*st));
    st->grid = *grid;
    for (int k = d; k < 3; ++k) { st->grid.M[k] = 1; st->grid.lo[k] = 0.0; st->grid.h[k] = 1.0; }
    st->d = d;
    st->dtype = dtype;
    st->n = n;
    st->m = m;
    st->ncells = ncell;
    st->nprobes = np;
    st->probe_seed = opts ? opts->probe_seed : 0;
    cudaGetDevice(&st->device);
    const size_t es = dtype == FKSKI_F32 ? 4 : 8;
    const int64_t nb = ipow(7, d);
    int rc = FKSKI_OK;
    if (pool_alloc(&st->band, es * nb * m, s) != FKSKI_OK || pool_alloc(&st->wty, es * m, s) != FKSKI_OK ||
        (np > 0 && pool_alloc(&st->wtz, es * np * m, s) != FKSKI_OK))
        rc = FKSKI_E_OOM;
    if (rc == FKSKI_OK) {
        if (dtype == FKSKI_F32) {
            const float *Xf = (const float *)X, *yf = (const float *)y, *Zf = (const float *)Z;
            rc = d == 1 ? precompute_typed<float, 1>(st, Xf, yf, Zf, opts, s)
               : d == 2 ? precompute_typed<float, 2>(st, Xf, yf, Zf, opts, s)
                        : precompute_typed<float, 3>(st, Xf, yf, Zf, opts, s);
        } else {
            const double *Xd = (const double *)X, *yd = (const double *)y, *Zd = (const double *)Z;
            rc = d == 1 ? precompute_typed<double, 1>(st, Xd, yd, Zd, opts, s)
               : d == 2 ? precompute_typed<double, 2>(st, Xd, yd, Zd, opts, s)
                        : precompute_typed<double, 3>(st, Xd, yd, Zd, opts, s);
        }
    }
    if (rc != FKSKI_OK) {
        cudaStreamSynchronize(s);
        destroy_stats(st);
        return rc;
    }
    *out = st;
    return FKSKI_OK;
}

}  // namespace fk
