// K_G = K_UU on the regular grid: multilevel Toeplitz (Sec. 2.2, "SKI running time"), applied
// through circulant embedding and FFTs (Lee 1986) in shared memory.
//
// RBF ARD factorises over axes, K_G = s T_1 (x) ... (x) T_d with T_k the symmetric Toeplitz
// matrix of exp(-1/2 (delta h_k / l_k)^2): one batched pass per axis, each line zero-padded to
// L_k = 2^ceil(log2(2 M_k - 1)), transformed, scaled by the real spectrum of the embedded
// circulant, transformed back and cropped.  Two real lines ride in one complex FFT (real and
// imaginary parts): the spectrum of a symmetric real circulant is real, so the two never mix.
//
// Matern-5/2 is not separable: the d-level embedding of k(delta_1 h_1, ..., delta_d h_d) on the
// L_1 x ... x L_d torus has a real spectrum; vectors are packed in pairs into complex tensors and
// transformed axis by axis (only the M-extent lines are transformed along each axis).
//
// FFT scheme: decimation in frequency (natural order in, bit-reversed out), the pointwise
// spectrum multiply in bit-reversed order, decimation in time back (bit-reversed in, natural out)
// -- no permutation pass.  Stages run in radix-4 groups (three twiddle products per group, the
// factors of -i exact) with one radix-2 stage when log2 L is odd.  Twiddles come from sincospi
// on the device.
#include "fkski_internal.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace fk {

template <typename T>
struct Cx;
template <>
struct Cx<float> { using t = float2; };
template <>
struct Cx<double> { using t = double2; };
template <>
struct Cx<dfl> { using t = dfl2; };

template <typename T>
__device__ __forceinline__ void sincospi_t(T x, T *s, T *c);
template <>
__device__ __forceinline__ void sincospi_t<float>(float x, float *s, float *c) { sincospif(x, s, c); }
template <>
__device__ __forceinline__ void sincospi_t<double>(double x, double *s, double *c) { sincospi(x, s, c); }

constexpr int FFT_T = 256;
constexpr int FFT_SMEM_CPLX = 4096;  // complex values of line data per CTA

template <typename T>
__device__ __forceinline__ void make_twiddles(typename Cx<T>::t *tw, int L) {
    // tw[k] = exp(-2 pi i k / L), k < L/2
    for (int k = threadIdx.x; k < L / 2; k += blockDim.x) {
        T s, c;
        sincospi_t<T>(T(2) * (T)k / (T)L, &s, &c);
        tw[k].x = c;
        tw[k].y = -s;
    }
}
// Double-float twiddles: the FP64 values rounded once to double-float.
template <>
__device__ __forceinline__ void make_twiddles<dfl>(dfl2 *tw, int L) {
    for (int k = threadIdx.x; k < L / 2; k += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)L, &s, &c);
        tw[k].x = dfl(c);
        tw[k].y = dfl(-s);
    }
}

// Butterfly arithmetic with every rounding spelled out (no contraction left to the compiler): a
// result depends on the transform length only, never on the launch shape the tuner picks.
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ dfl r_add(dfl a, dfl b) { return a + b; }
__device__ __forceinline__ dfl r_sub(dfl a, dfl b) { return a - b; }
__device__ __forceinline__ dfl r_mul(dfl a, dfl b) { return a * b; }
__device__ __forceinline__ dfl r_fma(dfl a, dfl b, dfl c) { return a * b + c; }
// a b + c d: for FP32 and FP64 exactly fma(a, b, c d) as written out before; double-float fuses
// the two products and the sum into one normalisation (df_dot2)
__device__ __forceinline__ float r_dot2(float a, float b, float c, float d) { return r_fma(a, b, r_mul(c, d)); }
__device__ __forceinline__ double r_dot2(double a, double b, double c, double d) { return r_fma(a, b, r_mul(c, d)); }
__device__ __forceinline__ dfl r_dot2(dfl a, dfl b, dfl c, dfl d) { return df_dot2(a, b, c, d); }

// DIF butterfly: (u, v) -> (u + v, (u - v) w)
template <typename C>
__device__ __forceinline__ void bf_dif(C &u, C &v, const C w) {
    const auto dx = r_sub(u.x, v.x), dy = r_sub(u.y, v.y);
    u.x = r_add(u.x, v.x);
    u.y = r_add(u.y, v.y);
    v.x = r_dot2(dx, w.x, -dy, w.y);
    v.y = r_dot2(dx, w.y, dy, w.x);
}

// DIT inverse butterfly: t = v conj(w); (u, v) -> (u + t, u - t)
template <typename C>
__device__ __forceinline__ void bf_dit(C &u, C &v, const C w) {
    const auto tx = r_dot2(v.x, w.x, v.y, w.y);
    const auto ty = r_dot2(v.y, w.x, -v.x, w.y);
    v.x = r_sub(u.x, tx);
    v.y = r_sub(u.y, ty);
    u.x = r_add(u.x, tx);
    u.y = r_add(u.y, ty);
}

// W_L^e for 0 <= e < L from the half table (W_L^{e + L/2} = -W_L^e)
template <typename C>
__device__ __forceinline__ C tw_at(const C *tw, int e, int L) {
    C w = tw[e & ((L >> 1) - 1)];
    if (e >= (L >> 1)) { w.x = -w.x; w.y = -w.y; }
    return w;
}
template <typename C>
__device__ __forceinline__ C cprod(const C a, const C w) {  // a w
    C r;
    r.x = r_dot2(a.x, w.x, -a.y, w.y);
    r.y = r_dot2(a.x, w.y, a.y, w.x);
    return r;
}
template <typename C>
__device__ __forceinline__ C cprodc(const C a, const C w) {  // a conj(w)
    C r;
    r.x = r_dot2(a.x, w.x, a.y, w.y);
    r.y = r_dot2(a.y, w.x, -a.x, w.y);
    return r;
}

// The butterfly of the radix-2 span-1 stages, whose twiddle is W^0 = 1: the product is exact,
// so it is left out (same values; a zero may change sign).
template <typename C>
__device__ __forceinline__ void bf_sum_dif(C &u, C &v) {  // (u, v) -> (u + v, u - v)
    const auto dx = r_sub(u.x, v.x), dy = r_sub(u.y, v.y);
    u.x = r_add(u.x, v.x);
    u.y = r_add(u.y, v.y);
    v.x = dx;
    v.y = dy;
}

// Shared-memory line layout.  PAD inserts one complex slot after every 8, so that the small-span
// stages, whose four accesses of a group lie at a stride of 2 to 8 slots, spread over all banks
// instead of a quarter of them; lines are then L + L/8 slots apart.
template <bool PAD>
__device__ __forceinline__ int pad_index(int e) { return PAD ? e + (e >> 3) : e; }
template <bool PAD>
__host__ __device__ __forceinline__ int line_stride(int L) { return PAD ? L + (L >> 3) : L; }

// In-place DIF over `nl` lines of length L stored contiguously (line stride L), natural order in,
// bit-reversed out.  RADIX 4 runs two radix-2 stages (spans h, h/2) per pass over shared memory:
// each thread keeps 4 values in registers, halving the passes and barriers.  The stages run from
// span h0 down to 1 (h0 = L/2 for a whole transform; a caller that has already done the larger
// spans passes the next one).
template <typename T, int RADIX, bool PAD = false>
__device__ __forceinline__ void fft_dif(typename Cx<T>::t *x, int nl, int L, const typename Cx<T>::t *tw, int h0 = 0) {
    using C = typename Cx<T>::t;
    const int LS = line_stride<PAD>(L);
    auto at = [&](int line, int e) -> C & { return x[line * LS + pad_index<PAD>(e)]; };
    int h = h0 > 0 ? h0 : (L >> 1);
    if (RADIX == 4) {
        const int ng = nl * (L >> 2);
        const int lq = __ffs(L) - 3;  // log2(L/4)
        for (; h >= 2; h >>= 2) {
            const int q = h >> 1, lqq = __ffs(q) - 1;
            const int tA = L / (2 * h), tB = L / h;
            for (int b = threadIdx.x; b < ng; b += blockDim.x) {
                const int line = b >> lq, k = b & ((L >> 2) - 1);
                const int j = k & (q - 1), blk = k >> lqq;
                const int e0 = blk * 2 * h + j;
                const C a0 = at(line, e0), a1 = at(line, e0 + q), a2 = at(line, e0 + h), a3 = at(line, e0 + h + q);
                // spans h and h/2 at once: with w = W^(j tA), W^((j+q) tA) = -i w and W^(j tB) = w^2,
                //   out0 = s + t, out1 = (s - t) w^2, out2 = (d - i e) w, out3 = (d + i e) w^3
                // for s = a0 + a2, t = a1 + a3, d = a0 - a2, e = a1 - a3
                C sv, tv, d, e;
                sv.x = r_add(a0.x, a2.x); sv.y = r_add(a0.y, a2.y);
                tv.x = r_add(a1.x, a3.x); tv.y = r_add(a1.y, a3.y);
                d.x = r_sub(a0.x, a2.x); d.y = r_sub(a0.y, a2.y);
                e.x = r_sub(a1.x, a3.x); e.y = r_sub(a1.y, a3.y);
                C o0, o1, o2, o3;
                o0.x = r_add(sv.x, tv.x); o0.y = r_add(sv.y, tv.y);
                o1.x = r_sub(sv.x, tv.x); o1.y = r_sub(sv.y, tv.y);
                o2.x = r_add(d.x, e.y); o2.y = r_sub(d.y, e.x);
                o3.x = r_sub(d.x, e.y); o3.y = r_add(d.y, e.x);
                if (j > 0) {
                    o1 = cprod(o1, tw[j * tB]);
                    o2 = cprod(o2, tw[j * tA]);
                    o3 = cprod(o3, tw_at(tw, 3 * j * tA, L));
                }
                at(line, e0) = o0;
                at(line, e0 + q) = o1;
                at(line, e0 + h) = o2;
                at(line, e0 + h + q) = o3;
            }

            __syncthreads();
        }
    }
    const int nbf = nl * (L >> 1);
    const int lhalf = __ffs(L) - 2;  // log2(L/2)
    for (; h >= 1; h >>= 1) {
        const int tstep = L / (2 * h);
        const int lh = __ffs(h) - 1;
        for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
            const int line = b >> lhalf, k = b & ((L >> 1) - 1);
            const int j = k & (h - 1), blk = k >> lh;
            const int e0 = blk * 2 * h + j;
            C u = at(line, e0), v = at(line, e0 + h);
            if (h == 1)
                bf_sum_dif(u, v);
            else
                bf_dif(u, v, tw[j * tstep]);
            at(line, e0) = u;
            at(line, e0 + h) = v;
        }
        __syncthreads();
    }
}

// In-place DIT inverse (conjugate twiddles, no 1/L: folded into the spectrum), bit-reversed in,
// natural out.  RADIX 4 groups the spans (h, 2h) from h = 1 upwards.  Only the spans below htop
// run (htop = L for a whole transform; a caller that finishes the largest span itself passes L/2).
// With `lam`, the inputs of the first stage are first multiplied by lam[position in the line]
// (the pointwise spectrum product, rounded exactly as a separate pass would round it).
template <typename T, int RADIX, bool PAD = false>
__device__ __forceinline__ void fft_dit_inv(typename Cx<T>::t *x, int nl, int L, const typename Cx<T>::t *tw,
                                            int htop = 0, const T *__restrict__ lam = nullptr) {
    using C = typename Cx<T>::t;
    const int LS = line_stride<PAD>(L);
    auto at = [&](int line, int e) -> C & { return x[line * LS + pad_index<PAD>(e)]; };
    if (htop <= 0) htop = L;
    int h = 1;
    if (RADIX == 4) {
        const int ng = nl * (L >> 2);
        const int lq = __ffs(L) - 3;  // log2(L/4)
        for (; 4 * h <= htop; h <<= 2) {
            const int lh = __ffs(h) - 1;
            const int tA = L / (2 * h), tB = L / (4 * h);
            for (int b = threadIdx.x; b < ng; b += blockDim.x) {
                const int line = b >> lq, k = b & ((L >> 2) - 1);
                const int j = k & (h - 1), blk = k >> lh;
                const int e0 = blk * 4 * h + j;
                C a0 = at(line, e0), a1 = at(line, e0 + h), a2 = at(line, e0 + 2 * h), a3 = at(line, e0 + 3 * h);
                if (lam && h == 1) {
                    const T *lb = lam + blk * 4;
                    const T l0 = lb[0], l1 = lb[1], l2 = lb[2], l3 = lb[3];
                    a0.x = r_mul(a0.x, l0); a0.y = r_mul(a0.y, l0);
                    a1.x = r_mul(a1.x, l1); a1.y = r_mul(a1.y, l1);
                    a2.x = r_mul(a2.x, l2); a2.y = r_mul(a2.y, l2);
                    a3.x = r_mul(a3.x, l3); a3.y = r_mul(a3.y, l3);
                }
                // spans h and 2h at once: with v = W^(j tB), W^(j tA) = v^2 and W^((j+h) tB) = -i v,
                //   b1 = a1 conj(v^2), b2 = a2 conj(v), b3 = a3 conj(v^3);
                //   out0 = s + t, out2 = s - t, out1 = d + i e, out3 = d - i e
                // for s = a0 + b1, t = b2 + b3, d = a0 - b1, e = b2 - b3
                if (j > 0) {
                    a1 = cprodc(a1, tw[j * tA]);
                    a2 = cprodc(a2, tw[j * tB]);
                    a3 = cprodc(a3, tw_at(tw, 3 * j * tB, L));
                }
                C sv, tv, d, e;
                sv.x = r_add(a0.x, a1.x); sv.y = r_add(a0.y, a1.y);
                d.x = r_sub(a0.x, a1.x); d.y = r_sub(a0.y, a1.y);
                tv.x = r_add(a2.x, a3.x); tv.y = r_add(a2.y, a3.y);
                e.x = r_sub(a2.x, a3.x); e.y = r_sub(a2.y, a3.y);
                a0.x = r_add(sv.x, tv.x); a0.y = r_add(sv.y, tv.y);
                a2.x = r_sub(sv.x, tv.x); a2.y = r_sub(sv.y, tv.y);
                a1.x = r_sub(d.x, e.y); a1.y = r_add(d.y, e.x);
                a3.x = r_add(d.x, e.y); a3.y = r_sub(d.y, e.x);
                at(line, e0) = a0;
                at(line, e0 + h) = a1;
                at(line, e0 + 2 * h) = a2;
                at(line, e0 + 3 * h) = a3;
            }
            __syncthreads();
        }
    }
    const int nbf = nl * (L >> 1);
    const int lhalf = __ffs(L) - 2;  // log2(L/2)
    for (; h < htop; h <<= 1) {
        const int tstep = L / (2 * h);
        const int lh = __ffs(h) - 1;
        for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
            const int line = b >> lhalf, k = b & ((L >> 1) - 1);
            const int j = k & (h - 1), blk = k >> lh;
            const int e0 = blk * 2 * h + j;
            C u = at(line, e0), v = at(line, e0 + h);
            if (lam && h == 1) {
                const T lu = lam[blk * 2], lv = lam[blk * 2 + 1];
                u.x = r_mul(u.x, lu); u.y = r_mul(u.y, lu);
                v.x = r_mul(v.x, lv); v.y = r_mul(v.y, lv);
            }
            if (h == 1)
                bf_sum_dif(u, v);
            else
                bf_dit(u, v, tw[j * tstep]);
            at(line, e0) = u;
            at(line, e0 + h) = v;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ Kronecker (real) axis pass
// Vector layout per rhs: [O][M][S] (axis of length M, S = product of later axes).
// Real lines l = (r*O + o)*S + s; two consecutive lines form one complex line.
// Lines of different right-hand sides never share a complex transform: FP32 rounding in the
// shared transform is relative to the larger of the two lines, which would put errors of one
// vector's size into the other.  When a rhs has an odd number of lines, its last line is paired
// with an empty padding line (index space per rhs rounded up to even).
struct RealPass {
    int64_t nlines;  // R * lpr2 (padded line slots)
    int64_t lpr;     // real lines per rhs = O * S
    int64_t lpr2;    // lpr rounded up to even
    int64_t S;       // inner stride
    int M, L;
    int Q;           // real lines per CTA (even)
};

constexpr int FFT_TMAX = 512;

// One CTA transforms Q real lines (Q/2 complex lines).  Shared memory: the twiddles (copied from
// a table computed once per operator), the Q line base addresses (the only 64-bit index
// arithmetic, once per line), then the lines in the padded layout (pad_index).  Two stages are
// folded into the global-memory
// phases: the upper half of every embedded line is zero (M <= L/2), so the first DIF stage (span
// L/2) is one complex multiply at load time, and only the first M outputs are kept, so the last
// DIT stage (span L/2) is one complex multiply-add at store time.  The spectrum product is folded
// into the first DIT stage.
template <typename T, bool EPI, int RADIX>
__global__ void __launch_bounds__(FFT_TMAX) k_kron_pass(const T *__restrict__ in, T *__restrict__ out, RealPass p,
                                                      const T *__restrict__ lam_br,
                                                      const typename Cx<T>::t *__restrict__ tw_g,
                                                      const T *__restrict__ addv,
                                                      const double *__restrict__ alpha_dev, double alpha_host,
                                                      const int *__restrict__ gate) {
    if (gate && *gate) return;
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int L = p.L, M = p.M, Q = p.Q, H = L >> 1;
    const int LS = line_stride<true>(L);
    const int nc = Q >> 1;
    C *tw = reinterpret_cast<C *>(smraw);
    long long *la = reinterpret_cast<long long *>(tw + H);
    C *x = reinterpret_cast<C *>(la + Q);
    for (int k = threadIdx.x; k < H; k += blockDim.x) tw[k] = tw_g[k];
    const int64_t l0 = (int64_t)blockIdx.x * Q;
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
        // real line slot -> base address of its first element (-1: padding slot or past the end)
        const int64_t slot = l0 + q;
        long long a = -1;
        if (slot < p.nlines) {
            const int64_t lr = slot % p.lpr2;
            if (lr < p.lpr) {
                const int64_t l = (slot / p.lpr2) * p.lpr + lr;
                a = (l / p.S) * (int64_t)M * p.S + (l % p.S);
            }
        }
        la[q] = a;
    }
    __syncthreads();
    const int64_t S = p.S;
    const int lc = __ffs(nc) - 1;  // nc is a power of two
    // load complex line c, element i < L/2 (real parts: line 2c, imaginary: line 2c+1), and apply
    // the first DIF stage against the zero upper half: (u, 0) -> (u, u w_i)
    auto load_one = [&](int c, int i) {
        const long long a0 = la[2 * c], a1 = la[2 * c + 1];
        C u;
        u.x = T(0);
        u.y = T(0);
        if (i < M) {
            if (a0 >= 0) u.x = in[a0 + (int64_t)i * S];
            if (a1 >= 0) u.y = in[a1 + (int64_t)i * S];
        }
        const C w = tw[i];
        C v;
        v.x = r_dot2(u.x, w.x, -u.y, w.y);
        v.y = r_dot2(u.x, w.y, u.y, w.x);
        x[c * LS + pad_index<true>(i)] = u;
        x[c * LS + pad_index<true>(i + H)] = v;
    };
    if (S == 1) {  // lines are contiguous: consecutive threads along the line (H is a power of two)
        const int lh = __ffs(H) - 1;
        for (int e = threadIdx.x; e < nc * H; e += blockDim.x) load_one(e >> lh, e & (H - 1));
    } else {  // lines are neighbours in memory: consecutive threads across lines
        for (int e = threadIdx.x; e < nc * H; e += blockDim.x) load_one(e & (nc - 1), e >> lc);
    }
    __syncthreads();
    fft_dif<T, RADIX, true>(x, nc, L, tw, H >> 1);
    fft_dit_inv<T, RADIX, true>(x, nc, L, tw, H, lam_br);
    const T alpha = EPI ? (alpha_dev ? (T)(*alpha_dev) : (T)alpha_host) : T(0);
    // last DIT stage (span L/2) for the kept outputs i < M: u + v conj(w_i)
    auto store_one = [&](int c, int i) {
        const C u = x[c * LS + pad_index<true>(i)], v = x[c * LS + pad_index<true>(i + H)], w = tw[i];
        const T tx = r_dot2(v.x, w.x, v.y, w.y);
        const T ty = r_dot2(v.y, w.x, -v.x, w.y);
        const long long a0 = la[2 * c], a1 = la[2 * c + 1];
        if (a0 >= 0) {
            const int64_t a = a0 + (int64_t)i * S;
            T r = r_add(u.x, tx);
            if (EPI) r = fma(alpha, addv[a], r);
            out[a] = r;
        }
        if (a1 >= 0) {
            const int64_t a = a1 + (int64_t)i * S;
            T r = r_add(u.y, ty);
            if (EPI) r = fma(alpha, addv[a], r);
            out[a] = r;
        }
    };
    if (S == 1) {
        const int lh = __ffs(H) - 1;
        for (int e = threadIdx.x; e < nc * H; e += blockDim.x)
            if ((e & (H - 1)) < M) store_one(e >> lh, e & (H - 1));
    } else {
        for (int e = threadIdx.x; e < nc * M; e += blockDim.x) store_one(e & (nc - 1), e >> lc);
    }
}

// ------------------------------------------------------------------ register FFT pass (L <= 256)
// The same embedded Toeplitz product along one axis, with each complex line's transform held in
// registers: L = L1 * L2 (L2 <= L1 <= 16) and the four-step decomposition
//   X[k1 + L1 k2] = sum_{n2} W_L2^{n2 k2} W_L^{n2 k1} sum_{n1} x[L2 n1 + n2] W_L1^{n1 k1}:
// L1 threads per line; thread n2 runs the L1-point DFT of its column, applies W_L^{n2 k1}, and
// the line's threads exchange through shared memory (one warp-synchronous transpose) so that
// thread k1 holds X[k1 + L1 k2] for all k2 after its L2-point DFT.  The spectrum product and the
// inverse run the same steps backwards, so a line needs two transposes and no block barrier;
// the block only synchronises around the coalesced load and store of its lines.  The exchange
// rows are padded to L2 + 1 complex values (conflict-free transposes).  Lines never interact,
// so results do not depend on how many lines a CTA holds (the tuner's only choice here).
template <typename C>
__device__ __forceinline__ C cmul(const C a, const C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C>
__device__ __forceinline__ C cmulc(const C a, const C b) {  // a * conj(b)
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
// double-float: each part as one fused a b + c d
__device__ __forceinline__ dfl2 cmul(const dfl2 a, const dfl2 b) {
    dfl2 r;
    r.x = df_dot2(a.x, b.x, -a.y, b.y);
    r.y = df_dot2(a.x, b.y, a.y, b.x);
    return r;
}
__device__ __forceinline__ dfl2 cmulc(const dfl2 a, const dfl2 b) {
    dfl2 r;
    r.x = df_dot2(a.x, b.x, a.y, b.y);
    r.y = df_dot2(a.y, b.x, -a.x, b.y);
    return r;
}

// In-register DFT of size N (natural order in and out): radix-2 DIF, then the bit-reversal
// permutation as register renaming.  W_N^t = tw[t * (L / N)] (tw: exp(-2 pi i k / L), k < L/2);
// INV uses conjugate twiddles.
template <typename T, int N, int L, bool INV>
__device__ __forceinline__ void reg_dft(typename Cx<T>::t (&v)[N], const typename Cx<T>::t *tw) {
    using C = typename Cx<T>::t;
#pragma unroll
    for (int h = N / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int b0 = 0; b0 < N; b0 += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const C a = v[b0 + j], b = v[b0 + j + h];
                C sum, dif;
                sum.x = a.x + b.x; sum.y = a.y + b.y;
                dif.x = a.x - b.x; dif.y = a.y - b.y;
                v[b0 + j] = sum;
                const int t = j * (N / (2 * h));  // W_N^t
                if (t == 0) {
                    v[b0 + j + h] = dif;
                } else if (4 * t == N) {  // W = -i (forward) or +i (inverse)
                    C r;
                    if (INV) { r.x = -dif.y; r.y = dif.x; } else { r.x = dif.y; r.y = -dif.x; }
                    v[b0 + j + h] = r;
                } else {
                    const C w = tw[t * (L / N)];
                    v[b0 + j + h] = INV ? cmulc(dif, w) : cmul(dif, w);
                }
            }
        }
    }
    // bit-reversed -> natural
    C o[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int r = 0;
#pragma unroll
        for (int b = 1, q = k; b < N; b <<= 1, q >>= 1) r = (r << 1) | (q & 1);
        o[r] = v[k];
    }
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = o[k];
}

// W_L^e for any integer e >= 0 from the half table (W_L^{e + L/2} = -W_L^e); conjugated for INV.
template <typename T, int L, bool INV>
__device__ __forceinline__ typename Cx<T>::t tw_any(const typename Cx<T>::t *tw, int e) {
    e &= L - 1;
    typename Cx<T>::t w = tw[e & (L / 2 - 1)];
    if (e >= L / 2) { w.x = -w.x; w.y = -w.y; }
    if (INV) w.y = -w.y;
    return w;
}

template <typename T, bool EPI, int L1, int L2>
__global__ void __launch_bounds__(256) k_kron_pass_reg(const T *__restrict__ in, T *__restrict__ out, RealPass p,
                                                        const T *__restrict__ lam_br,
                                                        const typename Cx<T>::t *__restrict__ tw_g,
                                                        const T *__restrict__ addv,
                                                        const double *__restrict__ alpha_dev, double alpha_host,
                                                        const int *__restrict__ gate) {
    if (gate && *gate) return;
    using C = typename Cx<T>::t;
    constexpr int L = L1 * L2, H = L / 2;
    constexpr int LS = L + L1;  // per-line shared stride (complex): exchange rows of L2 + 1
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = p.M, Q = p.Q;
    const int nc = Q >> 1;
    C *tw = reinterpret_cast<C *>(smraw);
    T *lam = reinterpret_cast<T *>(tw + H);
    long long *la = reinterpret_cast<long long *>(lam + L + (L & 1));
    C *x = reinterpret_cast<C *>(la + Q);
    for (int k = threadIdx.x; k < H; k += blockDim.x) tw[k] = tw_g[k];
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        // natural-order spectrum from the bit-reversed table
        constexpr int LB = (L1 == 16 ? 4 : (L1 == 8 ? 3 : (L1 == 4 ? 2 : 1))) + (L2 == 16 ? 4 : (L2 == 8 ? 3 : (L2 == 4 ? 2 : 1)));
        lam[k] = lam_br[__brev((unsigned)k) >> (32 - LB)];
    }
    const int64_t l0 = (int64_t)blockIdx.x * Q;
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
        const int64_t slot = l0 + q;
        long long a = -1;
        if (slot < p.nlines) {
            const int64_t lr = slot % p.lpr2;
            if (lr < p.lpr) {
                const int64_t l = (slot / p.lpr2) * p.lpr + lr;
                a = (l / p.S) * (int64_t)M * p.S + (l % p.S);
            }
        }
        la[q] = a;
    }
    __syncthreads();
    const int64_t S = p.S;
    const int lc = __ffs(nc) - 1;  // nc is a power of two
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // coalesced load of the data part (i < M) of every line: real parts line 2c, imaginary 2c+1
    auto load_one = [&](int c, int i) {
        const long long a0 = la[2 * c], a1 = la[2 * c + 1];
        C u;
        u.x = a0 >= 0 ? in[a0 + (int64_t)i * S] : T(0);
        u.y = a1 >= 0 ? in[a1 + (int64_t)i * S] : T(0);
        x[c * LS + i] = u;
    };
    if (S == 1) {  // consecutive threads along the line (H = L / 2 >= M, a power of two)
        for (int e = threadIdx.x; e < nc * H; e += blockDim.x)
            if ((e & (H - 1)) < M) load_one(e / H, e & (H - 1));
    } else {
        for (int e = threadIdx.x; e < nc * M; e += blockDim.x) load_one(e & (nc - 1), e >> lc);
    }
    __syncthreads();
    // one line per group of L1 lanes; the loop over a warp's lines is warp-uniform (the
    // exchanges synchronise the whole warp), idle groups only take part in the syncs
    constexpr int GPW = 32 / L1;
    const int j = lane % L1;
    for (int cb = warp * GPW; cb < nc; cb += nw * GPW) {
        const int c = cb + lane / L1;
        const bool act = c < nc;
        C *xl = x + (act ? c : 0) * LS;
        const bool col = act && j < L2;  // thread owns column n2 = j in the outer steps
        // forward, step 1: DFT over n1 of x[L2 n1 + j] (zero beyond M), then W_L^{j k1}
        C v[L1];
        if (col) {
#pragma unroll
            for (int n1 = 0; n1 < L1; ++n1) {
                const int n = L2 * n1 + j;
                if (n < M) v[n1] = xl[n];
                else { v[n1].x = T(0); v[n1].y = T(0); }
            }
            reg_dft<T, L1, L, false>(v, tw);
#pragma unroll
            for (int k1 = 1; k1 < L1; ++k1) v[k1] = cmul(v[k1], tw_any<T, L, false>(tw, j * k1));
        }
        __syncwarp();
        if (col) {
#pragma unroll
            for (int k1 = 0; k1 < L1; ++k1) xl[k1 * (L2 + 1) + j] = v[k1];
        }
        __syncwarp();
        // step 2: thread k1 = j: DFT over n2 -> X[k1 + L1 k2]; spectrum; inverse over k2;
        // then W_L^{-n2 k1}
        if (act) {
            C u[L2];
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) u[n2] = xl[j * (L2 + 1) + n2];
            reg_dft<T, L2, L, false>(u, tw);
#pragma unroll
            for (int k2 = 0; k2 < L2; ++k2) {
                const T lm = lam[j + L1 * k2];
                u[k2].x *= lm;
                u[k2].y *= lm;
            }
            reg_dft<T, L2, L, true>(u, tw);
#pragma unroll
            for (int n2 = 1; n2 < L2; ++n2) u[n2] = cmul(u[n2], tw_any<T, L, true>(tw, n2 * j));
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) xl[j * (L2 + 1) + n2] = u[n2];
        }
        __syncwarp();
        // inverse, step 1 backwards: thread n2 = j: inverse DFT over k1 -> y[L2 n1 + j]
        if (col) {
#pragma unroll
            for (int k1 = 0; k1 < L1; ++k1) v[k1] = xl[k1 * (L2 + 1) + j];
            reg_dft<T, L1, L, true>(v, tw);
        }
        __syncwarp();
        if (col) {
#pragma unroll
            for (int n1 = 0; n1 < L1; ++n1) {
                const int n = L2 * n1 + j;
                if (n < M) xl[n] = v[n1];
            }
        }
        __syncwarp();
    }
    __syncthreads();
    const T alpha = EPI ? (alpha_dev ? (T)(*alpha_dev) : (T)alpha_host) : T(0);
    auto store_one = [&](int c, int i) {
        const C u = x[c * LS + i];
        const long long a0 = la[2 * c], a1 = la[2 * c + 1];
        if (a0 >= 0) {
            const int64_t a = a0 + (int64_t)i * S;
            T r = u.x;
            if (EPI) r = fma(alpha, addv[a], r);
            out[a] = r;
        }
        if (a1 >= 0) {
            const int64_t a = a1 + (int64_t)i * S;
            T r = u.y;
            if (EPI) r = fma(alpha, addv[a], r);
            out[a] = r;
        }
    };
    if (S == 1) {
        for (int e = threadIdx.x; e < nc * H; e += blockDim.x)
            if ((e & (H - 1)) < M) store_one(e / H, e & (H - 1));
    } else {
        for (int e = threadIdx.x; e < nc * M; e += blockDim.x) store_one(e & (nc - 1), e >> lc);
    }
}

// Twiddle table exp(-2 pi i k / L), k < L/2, for the Kronecker passes (same formula as the
// per-CTA tables, computed once per operator).
template <typename T>
__global__ void __launch_bounds__(FFT_T) k_twiddles(typename Cx<T>::t *__restrict__ tw, int L) {
    make_twiddles<T>(tw, L);
}

// ------------------------------------------------------------------ complex axis pass (BTTB)
// Complex tensor with lines along one axis: line l = o*S + s, input extent Min, output extent
// Mout along the axis (zero-pad to L on input, crop on output).  MODE 0: DIF forward,
// 1: DIT inverse, 2: DIF -> multiply by lam[(k)*S + s] (bit-reversed k) -> DIT.
struct CplxPass {
    int64_t nlines, S;
    int Min, Mout, L, Q;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(FFT_T) k_cplx_pass(const typename Cx<T>::t *__restrict__ in, typename Cx<T>::t *__restrict__ out,
                                                      CplxPass p, const T *__restrict__ lam, const int *__restrict__ gate) {
    if (gate && *gate) return;
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *tw = reinterpret_cast<C *>(smraw);
    C *x = tw + p.L / 2;
    const int L = p.L, Q = p.Q;
    make_twiddles<T>(tw, L);
    const int64_t l0 = (int64_t)blockIdx.x * Q;
    const int nq = (int)min((int64_t)Q, p.nlines - l0);
    const int64_t S = p.S;
    for (int e = threadIdx.x; e < Q * L; e += blockDim.x) {
        x[e].x = T(0);
        x[e].y = T(0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nq * p.Min; e += blockDim.x) {
        int q, i;
        if (S == 1) { q = e / p.Min; i = e % p.Min; } else { q = e % nq; i = e / nq; }
        const int64_t l = l0 + q;
        x[q * L + i] = in[(l / S) * (int64_t)p.Min * S + (l % S) + (int64_t)i * S];
    }
    __syncthreads();
    if (MODE == 0 || MODE == 2) fft_dif<T, 4>(x, Q, L, tw);
    if (MODE == 2) {
        for (int e = threadIdx.x; e < nq * L; e += blockDim.x) {
            const int q = e / L, k = e % L;
            const int64_t s = (l0 + q) % S;
            const T lm = lam[(int64_t)k * S + s];
            x[e].x *= lm;
            x[e].y *= lm;
        }
        __syncthreads();
    }
    if (MODE == 1 || MODE == 2) fft_dit_inv<T, 4>(x, Q, L, tw);
    for (int e = threadIdx.x; e < nq * p.Mout; e += blockDim.x) {
        int q, i;
        if (S == 1) { q = e / p.Mout; i = e % p.Mout; } else { q = e % nq; i = e / nq; }
        const int64_t l = l0 + q;
        out[(l / S) * (int64_t)p.Mout * S + (l % S) + (int64_t)i * S] = x[q * L + i];
    }
}

// real rhs into complex tensors of shape (M_1..M_d), one rhs each (imaginary part zero: rhs
// never share a transform, for the reason given at RealPass), and back (with epilogue)
template <typename T>
__global__ void k_pack_pairs(const T *__restrict__ v, typename Cx<T>::t *__restrict__ z, int64_t m, int nrhs,
                             const int *__restrict__ gate) {
    if (gate && *gate) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nrhs * m; e += (int64_t)gridDim.x * blockDim.x) {
        typename Cx<T>::t c;
        c.x = v[e];
        c.y = T(0);
        z[e] = c;
    }
}

template <typename T>
__global__ void k_unpack_pairs(const typename Cx<T>::t *__restrict__ z, T *__restrict__ out, int64_t m, int nrhs,
                               const T *__restrict__ addv, const double *__restrict__ alpha_dev, double alpha_host,
                               const int *__restrict__ gate) {
    if (gate && *gate) return;
    const T alpha = addv ? (alpha_dev ? (T)(*alpha_dev) : (T)alpha_host) : T(0);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nrhs * m; e += (int64_t)gridDim.x * blockDim.x) {
        T v = z[e].x;
        if (addv) v = fma(alpha, addv[e], v);
        out[e] = v;
    }
}

// ------------------------------------------------------------------ spectra
// First column of the embedded circulant along one axis of length L: c[i] = k(delta(i) h)
// with delta(i) = i for i < M, L - i for i > L - M, 0-weight slots otherwise.
__device__ __forceinline__ int circ_delta(int i, int M, int L, bool &valid) {
    if (i < M) { valid = true; return i; }
    if (i > L - M) { valid = true; return L - i; }
    valid = false;
    return 0;
}

// Kronecker factor spectrum (one CTA): lam_br[k] = scale / L * DFT(c)[bitrev(k)] for the RBF
// factor exp(-1/2 (delta h / l)^2) (or its derivative in l when deriv).  Always computed in FP64
// and rounded once to T: an FP32 transform would give the small eigenvalues absolute errors near
// 2^-24 of the largest, i.e. a different operator from the FP64 one, and the FP32 solver's
// true-residual checks (FP64 K_G) must see the same operator as its iterations.
template <typename T>
__global__ void __launch_bounds__(FFT_T) k_spectrum_1d(T *__restrict__ lam_br, int M, int L, double h, double ell,
                                                        int deriv, double scale) {
    using C = double2;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *tw = reinterpret_cast<C *>(smraw);
    C *x = tw + L / 2;
    make_twiddles<double>(tw, L);
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        bool ok;
        const int dl = circ_delta(i, M, L, ok);
        double v = 0.0;
        if (ok) {
            const double r = (double)dl * h / ell;
            v = exp(-0.5 * r * r);
            if (deriv) v *= r * r / ell;
        }
        x[i].x = v;
        x[i].y = 0.0;
    }
    __syncthreads();
    fft_dif<double, 4>(x, 1, L, tw);
    for (int k = threadIdx.x; k < L; k += blockDim.x) lam_br[k] = (T)(scale / L * x[k].x);
}

// d-level embedding values for a (possibly derivative) stationary kernel, written as a complex
// tensor over the L-box (axis 0 outermost).  kind: 0 Matern-5/2, 1 RBF; deriv: -1 value,
// k in [0,d) d/dl_k, d -> d/ds.
struct EmbedParams {
    int d;
    int M[3], L[3];
    double h[3], ell[3];
    double s;
    int kind, deriv;
};

template <typename T>
__global__ void k_embed_values(typename Cx<T>::t *__restrict__ z, EmbedParams ep, int64_t N) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e;
        double q = 0.0;
        bool ok = true;
        double dk2[3] = {0, 0, 0};
        for (int k = ep.d - 1; k >= 0; --k) {
            const int i = (int)(r % ep.L[k]);
            r /= ep.L[k];
            bool v;
            const int dl = circ_delta(i, ep.M[k], ep.L[k], v);
            ok = ok && v;
            const double u = (double)dl * ep.h[k] / ep.ell[k];
            dk2[k] = u * u / ep.ell[k];
            q += u * u;
        }
        double val = 0.0;
        if (ok) {
            if (ep.kind == 0) {
                const double rr = sqrt(q), s5 = sqrt(5.0);
                if (ep.deriv < 0 || ep.deriv == ep.d)
                    val = (ep.deriv < 0 ? ep.s : 1.0) * (1.0 + s5 * rr + 5.0 / 3.0 * q) * exp(-s5 * rr);
                else
                    val = ep.s * (5.0 / 3.0) * (1.0 + s5 * rr) * exp(-s5 * rr) * dk2[ep.deriv];
            } else {
                val = (ep.deriv == ep.d ? 1.0 : ep.s) * exp(-0.5 * q);
                if (ep.deriv >= 0 && ep.deriv < ep.d) val *= dk2[ep.deriv];
            }
        }
        z[e].x = (T)val;
        z[e].y = T(0);
    }
}

template <typename T>
__global__ void k_take_real_scaled(const double2 *__restrict__ z, T *__restrict__ lam, int64_t N, double scale) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
        lam[e] = (T)(scale * (double)z[e].x);
}

// ------------------------------------------------------------------ operator object
struct KgOp {
    fkski_grid g;
    int d, dtype;
    int64_t m;
    int L[3];
    int kind;           // FKSKI_RBF / FKSKI_MATERN52
    int param;
    void *lam[3];       // Kronecker spectra (bit-reversed), L_k each
    void *tw[3];        // Kronecker pass twiddles, L_k / 2 complex each
    bool tw_ok[3];      // twiddle table written
    void *lamN;         // BTTB spectrum over the L-box (bit-reversed per axis)
    int64_t N;          // prod L_k
    void *scratch;      // work buffer
    size_t scratch_bytes;
    const int *gate;    // device flag: when set, the product's kernels return at once (null: always run)
};

static int next_pow2(int64_t v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

int kgop_create(const fkski_grid *grid, int dtype, KgOp **op) {
    *op = nullptr;
    KgOp *k = new KgOp;
    memset(k, 0, sizeof(*k));
    k->g = *grid;
    k->d = grid->d;
    k->dtype = dtype;
    k->m = 1;
    k->N = 1;
    k->kind = -1;
    for (int a = 0; a < k->d; ++a) {
        k->m *= grid->M[a];
        k->L[a] = next_pow2(2 * grid->M[a] - 1);
        if (k->L[a] > FFT_SMEM_CPLX) {
            delete k;
            return FKSKI_E_UNSUPPORTED;
        }
        k->N *= k->L[a];
    }
    *op = k;
    return FKSKI_OK;
}

void kgop_destroy(KgOp *op) {
    if (!op) return;
    for (int a = 0; a < 3; ++a) {
        if (op->lam[a]) cudaFree(op->lam[a]);
        if (op->tw[a]) cudaFree(op->tw[a]);
    }
    if (op->lamN) cudaFree(op->lamN);
    if (op->scratch) cudaFree(op->scratch);
    delete op;
}

static size_t esz(int dtype) { return dtype == FKSKI_F32 ? 4 : 8; }  // FP64 and double-float: 8

static int ensure(void **p, size_t &have, size_t want) {
    if (have >= want && *p) return FKSKI_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    have = 0;
    if (cudaMalloc(p, want) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return FKSKI_E_OOM;
    }
    have = want;
    return FKSKI_OK;
}

// Lines along axis a of a complex tensor whose extents are ext[0..d-1].
static CplxPass cplx_geom(const int64_t ext[3], int d, int a, int Min, int Mout, int L, int64_t nbatch) {
    CplxPass p;
    int64_t O = nbatch, S = 1;
    for (int k = 0; k < a; ++k) O *= ext[k];
    for (int k = a + 1; k < d; ++k) S *= ext[k];
    p.nlines = O * S;
    p.S = S;
    p.Min = Min;
    p.Mout = Mout;
    p.L = L;
    p.Q = std::max(1, FFT_SMEM_CPLX / L);
    return p;
}

template <typename T>
static int launch_cplx(const typename Cx<T>::t *in, typename Cx<T>::t *out, CplxPass p, int mode, const T *lam,
                       cudaStream_t s, const int *gate = nullptr) {
    using C = typename Cx<T>::t;
    const size_t sm = sizeof(C) * ((size_t)p.L / 2 + (size_t)p.Q * p.L);
    const unsigned nb = (unsigned)cdiv(p.nlines, p.Q);
    if (mode == 0) {
        FK_TRY(raise_smem_limit((const void *)k_cplx_pass<T, 0>, sm));
        k_cplx_pass<T, 0><<<nb, FFT_T, sm, s>>>(in, out, p, lam, gate);
    } else if (mode == 1) {
        FK_TRY(raise_smem_limit((const void *)k_cplx_pass<T, 1>, sm));
        k_cplx_pass<T, 1><<<nb, FFT_T, sm, s>>>(in, out, p, lam, gate);
    } else {
        FK_TRY(raise_smem_limit((const void *)k_cplx_pass<T, 2>, sm));
        k_cplx_pass<T, 2><<<nb, FFT_T, sm, s>>>(in, out, p, lam, gate);
    }
    FK_LAUNCH();
    return FKSKI_OK;
}

// BTTB spectrum: embed kernel values on the L-box, forward DIF along every axis (bit-reversed
// order per axis), keep the real part scaled by 1/N.
// Computed in FP64 for both operator precisions (see k_spectrum_1d), rounded once to T.
template <typename T>
static int bttb_spectrum(KgOp *op, const fkski_kernel *kern, int param, cudaStream_t s) {
    using C = double2;
    const int d = op->d;
    const int64_t N = op->N;
    size_t have = 0;
    if (!op->lamN) FK_TRY(ensure(&op->lamN, have, sizeof(T) * N));
    C *z0 = nullptr, *z1 = nullptr;
    FK_TRY(pool_alloc((void **)&z0, sizeof(C) * N, s));
    FK_TRY(pool_alloc((void **)&z1, sizeof(C) * N, s));
    EmbedParams ep;
    memset(&ep, 0, sizeof(ep));
    ep.d = d;
    for (int k = 0; k < d; ++k) {
        ep.M[k] = (int)op->g.M[k];
        ep.L[k] = op->L[k];
        ep.h[k] = op->g.h[k];
        ep.ell[k] = kern->lengthscale[k];
    }
    ep.s = kern->outputscale;
    ep.kind = kern->type == FKSKI_MATERN52 ? 0 : 1;
    ep.deriv = param;
    const unsigned nb = (unsigned)std::min<int64_t>(cdiv(N, 256), 4096);
    k_embed_values<double><<<nb, 256, 0, s>>>(z0, ep, N);
    FK_LAUNCH();
    int64_t ext[3] = {op->L[0], op->L[1], op->L[2]};
    C *cur = z0, *nxt = z1;
    for (int a = d - 1; a >= 0; --a) {
        CplxPass p = cplx_geom(ext, d, a, op->L[a], op->L[a], op->L[a], 1);
        FK_TRY(launch_cplx<double>(cur, nxt, p, 0, (const double *)nullptr, s));
        std::swap(cur, nxt);
    }
    k_take_real_scaled<T><<<nb, 256, 0, s>>>(cur, (T *)op->lamN, N, 1.0 / (double)N);
    FK_LAUNCH();
    cudaFreeAsync(z0, s);
    cudaFreeAsync(z1, s);
    return FKSKI_OK;
}

int kgop_set(KgOp *op, const fkski_kernel *kern, int param, cudaStream_t s) {
    if (!kern) return FKSKI_E_INVALID_ARG;
    if (kern->type != FKSKI_RBF && kern->type != FKSKI_MATERN52) return FKSKI_E_INVALID_ARG;
    if (param < -1 || param > op->d) return FKSKI_E_INVALID_ARG;
    for (int k = 0; k < op->d; ++k)
        if (!(kern->lengthscale[k] > 0.0) || !std::isfinite(kern->lengthscale[k])) return FKSKI_E_INVALID_ARG;
    if (!(kern->outputscale > 0.0)) return FKSKI_E_INVALID_ARG;
    op->kind = kern->type;
    op->param = param;
    const size_t es = esz(op->dtype);
    if (kern->type == FKSKI_RBF) {
        for (int a = 0; a < op->d; ++a) {
            size_t have = 0;
            if (!op->lam[a]) FK_TRY(ensure(&op->lam[a], have, es * op->L[a]));
            if (!op->tw[a]) {
                size_t have_tw = 0;
                FK_TRY(ensure(&op->tw[a], have_tw, es * op->L[a]));  // L/2 complex
            }
            if (!op->tw_ok[a]) {
                if (op->dtype == FKSKI_F32)
                    k_twiddles<float><<<1, FFT_T, 0, s>>>((float2 *)op->tw[a], op->L[a]);
                else if (op->dtype == FK_DF)
                    k_twiddles<dfl><<<1, FFT_T, 0, s>>>((dfl2 *)op->tw[a], op->L[a]);
                else
                    k_twiddles<double><<<1, FFT_T, 0, s>>>((double2 *)op->tw[a], op->L[a]);
                FK_LAUNCH();
                op->tw_ok[a] = true;
            }
            const double scale = (a == 0) ? (param == op->d ? 1.0 : kern->outputscale) : 1.0;
            const int deriv = (param == a) ? 1 : 0;
            const size_t sm = sizeof(double2) * ((size_t)op->L[a] / 2 + (size_t)op->L[a]);
            if (op->dtype == FKSKI_F32) {
                FK_TRY(raise_smem_limit((const void *)k_spectrum_1d<float>, sm));
                k_spectrum_1d<float><<<1, FFT_T, sm, s>>>((float *)op->lam[a], (int)op->g.M[a], op->L[a], op->g.h[a],
                                                          kern->lengthscale[a], deriv, scale);
            } else if (op->dtype == FK_DF) {
                FK_TRY(raise_smem_limit((const void *)k_spectrum_1d<dfl>, sm));
                k_spectrum_1d<dfl><<<1, FFT_T, sm, s>>>((dfl *)op->lam[a], (int)op->g.M[a], op->L[a], op->g.h[a],
                                                        kern->lengthscale[a], deriv, scale);
            } else {
                FK_TRY(raise_smem_limit((const void *)k_spectrum_1d<double>, sm));
                k_spectrum_1d<double><<<1, FFT_T, sm, s>>>((double *)op->lam[a], (int)op->g.M[a], op->L[a], op->g.h[a],
                                                           kern->lengthscale[a], deriv, scale);
            }
            FK_LAUNCH();
        }
        return FKSKI_OK;
    }
    if (op->dtype == FKSKI_F32) return bttb_spectrum<float>(op, kern, param, s);
    if (op->dtype == FK_DF) return bttb_spectrum<dfl>(op, kern, param, s);
    return bttb_spectrum<double>(op, kern, param, s);
}

// ------------------------------------------------------------------ pass configuration and tuner
// A Kronecker pass is launched with (kernel, complex lines per CTA, threads per CTA).  The choice
// changes speed only: lines are independent, and which kernel runs (register or shared-memory
// transform) depends on the precision and L alone.  The
// tuner times every candidate on the real pass shape (once per shape and process, outside any
// graph capture: the solver calls kgop_tune before capturing) and keeps the fastest; untuned shapes get a default that
// puts at least ~4 CTAs on every SM.
struct PassCfg {
    int radix, cl, threads;  // radix 0: the register kernel (k_kron_pass_reg)
    float ms;  // tuned time per launch (0: default, not tuned)
};

// Passes that run the register kernel (L = L1 * L2, L1 <= 16): FP32 up to L = 256; FP64 up to
// L = 64 (its 16-value columns need twice the registers, and for L = 128, 256 the
// shared-memory kernel is as fast or faster); double-float up to DF_REG_LMAX.  The rule depends
// on the shape only.
// L = 128, 256: the shared-memory radix-4 pass is faster (L = 256: 20.9 against 28.1 us per pass;
// L = 128, 17 rhs on a 64^3 grid: 1.71 against 1.85 ms per gradient iteration)
constexpr int DF_REG_LMAX = 64;
static bool reg_fft_ok(int dtype, int L) {
    return L >= 8 && L <= (dtype == FKSKI_F32 ? 256 : (dtype == FK_DF ? DF_REG_LMAX : 64));
}

struct PassKey {
    int dtype, L, M;
    int64_t S, nlines;
    bool operator<(const PassKey &o) const {
        if (dtype != o.dtype) return dtype < o.dtype;
        if (L != o.L) return L < o.L;
        if (M != o.M) return M < o.M;
        if (S != o.S) return S < o.S;
        return nlines < o.nlines;
    }
};

static std::mutex g_tune_mu;
static std::map<PassKey, PassCfg> g_tune;

static int device_sms() {
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

static PassCfg default_cfg(int dtype, const RealPass &p) {
    const int64_t ncl = p.nlines / 2;  // complex lines
    if (reg_fft_ok(dtype, p.L)) {
        int cl = 16;
        while (cl > 1 && cdiv(ncl, cl) < 4 * device_sms()) cl >>= 1;
        return PassCfg{0, cl, 128, 0.f};
    }
    int cl = std::max(1, FFT_SMEM_CPLX / p.L);
    while (cl > 1 && cdiv(ncl, cl) < 4 * device_sms()) cl >>= 1;
    return PassCfg{4, cl, 256, 0.f};
}

// Register-kernel shared memory: twiddles, natural-order spectrum, line addresses, padded lines.
template <typename T>
static size_t reg_pass_smem(int L, int cl) {
    const int L1 = L >= 128 ? 16 : (L >= 32 ? 8 : 4);
    return sizeof(typename Cx<T>::t) * ((size_t)L / 2 + (size_t)cl * (L + L1)) + sizeof(T) * (size_t)L +
           sizeof(long long) * 2 * (size_t)cl;
}

static PassCfg pass_config(int dtype, const RealPass &p, int nrhs) {
    (void)nrhs;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto it = g_tune.find(PassKey{dtype, p.L, p.M, p.S, p.nlines});
    return it != g_tune.end() ? it->second : default_cfg(dtype, p);
}

template <typename T>
static int launch_kron(const T *src, T *dst, RealPass p, const PassCfg &cfg, const T *lam,
                       const typename Cx<T>::t *tw, const T *addv, const double *alpha_dev, double alpha,
                       const int *gate, cudaStream_t s) {
    p.Q = 2 * cfg.cl;
    const unsigned nb = (unsigned)cdiv(p.nlines, p.Q);
    if (cfg.radix == 0) {
        const size_t smr = reg_pass_smem<T>(p.L, cfg.cl);
#define FK_KRONR(EPIV, A, B)                                                                                     \
    do {                                                                                                         \
        FK_TRY(raise_smem_limit((const void *)k_kron_pass_reg<T, EPIV, A, B>, smr));                           \
        k_kron_pass_reg<T, EPIV, A, B><<<nb, cfg.threads, smr, s>>>(src, dst, p, lam, tw, addv, alpha_dev, alpha, gate); \
    } while (0)
#define FK_KRONR_L(EPIV)                                     \
    switch (p.L) {                                           \
        case 8: FK_KRONR(EPIV, 4, 2); break;                 \
        case 16: FK_KRONR(EPIV, 4, 4); break;                \
        case 32: FK_KRONR(EPIV, 8, 4); break;                \
        case 64: FK_KRONR(EPIV, 8, 8); break;                \
        case 128: FK_KRONR(EPIV, 16, 8); break;              \
        case 256: FK_KRONR(EPIV, 16, 16); break;             \
        default: return FKSKI_E_UNSUPPORTED;                 \
    }
        if (addv) { FK_KRONR_L(true); } else { FK_KRONR_L(false); }
#undef FK_KRONR_L
#undef FK_KRONR
        FK_LAUNCH();
        return FKSKI_OK;
    }
    const size_t sm = sizeof(typename Cx<T>::t) * ((size_t)p.L / 2 + (size_t)cfg.cl * line_stride<true>(p.L)) +
                      sizeof(long long) * p.Q;
#define FK_KRON(EPIV, RADV)                                                                                      \
    do {                                                                                                         \
        FK_TRY(raise_smem_limit((const void *)k_kron_pass<T, EPIV, RADV>, sm)); \
        k_kron_pass<T, EPIV, RADV><<<nb, cfg.threads, sm, s>>>(src, dst, p, lam, tw, addv, alpha_dev, alpha, gate); \
    } while (0)
    if (addv) FK_KRON(true, 4); else FK_KRON(false, 4);
#undef FK_KRON
    FK_LAUNCH();
    return FKSKI_OK;
}

// Time the candidates of one pass shape on scratch data and record the fastest.
template <typename T>
static int tune_pass(int dtype, RealPass p, const T *lam, const typename Cx<T>::t *tw, T *buf_in, T *buf_out,
                     cudaStream_t s) {
    const PassKey key{dtype, p.L, p.M, p.S, p.nlines};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (g_tune.count(key)) return FKSKI_OK;
    }
    // Candidates are timed as a captured graph of TUNE_REPS launches on a private stream (the
    // per-launch host overhead would otherwise hide the kernels' differences).
    constexpr int TUNE_REPS = 10;
    cudaStream_t ts = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, ej = nullptr;
    FK_CUDA(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ej, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventRecord(ej, s);  // buffers were prepared on s
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ts, ej, 0);
    int rc = ce == cudaSuccess ? FKSKI_OK : note_cuda_error(ce, __FILE__, __LINE__);
    PassCfg best = default_cfg(dtype, p);
    best.ms = 1e30f;
    const int64_t ncl = std::max<int64_t>(1, p.nlines / 2);
    auto time_cfg = [&](const PassCfg &c) -> int {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal);
        int r = e == cudaSuccess ? FKSKI_OK : note_cuda_error(e, __FILE__, __LINE__);
        for (int k = 0; k < TUNE_REPS && r == FKSKI_OK; ++k)
            r = launch_kron<T>(buf_in, buf_out, p, c, lam, tw, nullptr, nullptr, 0.0, nullptr, ts);
        const cudaError_t ee = cudaStreamEndCapture(ts, &g);
        if (r != FKSKI_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        e = ee;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, ts);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, ts);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, ts);
        if (e == cudaSuccess) e = cudaEventRecord(e1, ts);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return note_cuda_error(e, __FILE__, __LINE__);
        ms /= TUNE_REPS;
        if (ms < best.ms) best = PassCfg{c.radix, c.cl, c.threads, ms};
        return FKSKI_OK;
    };
    if (reg_fft_ok(dtype, p.L)) {
        // register kernel only (its configurations are bit-identical to each other)
        for (int threads : {64, 128, 256}) {
            for (int cl = 1; cl <= 64 && rc == FKSKI_OK; cl <<= 1) {
                if (cl > 1 && cl / 2 >= ncl) break;
                if (reg_pass_smem<T>(p.L, cl) > 96 * 1024) break;
                rc = time_cfg(PassCfg{0, cl, threads, 0.f});
            }
        }
    } else {
        const int clmax = std::max(1, FFT_SMEM_CPLX / p.L);
        for (int radix : {4}) {
            for (int threads : {128, 256, 512}) {
                for (int cl = 1; cl <= clmax && rc == FKSKI_OK; cl <<= 1) {
                    if (cl > 1 && cl / 2 >= ncl) break;  // more lines per CTA than there are lines
                    rc = time_cfg(PassCfg{radix, cl, threads, 0.f});
                }
            }
        }
    }
    if (rc == FKSKI_OK) {
        ce = cudaEventRecord(ej, ts);  // s continues after the tuning launches
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, ej, 0);
        if (ce != cudaSuccess) rc = note_cuda_error(ce, __FILE__, __LINE__);
    }
    cudaStreamSynchronize(ts);
    cudaStreamDestroy(ts);
    if (ej) cudaEventDestroy(ej);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = best;
    return FKSKI_OK;
}

template <typename T>
static int kron_tune(KgOp *op, int nrhs, cudaStream_t s) {
    const int64_t m = op->m;
    T *buf = nullptr;
    FK_TRY(pool_alloc((void **)&buf, sizeof(T) * 2 * (size_t)nrhs * m, s));
    int rc = cudaMemsetAsync(buf, 0, sizeof(T) * 2 * (size_t)nrhs * m, s) == cudaSuccess ? FKSKI_OK : FKSKI_E_CUDA;
    for (int a = 0; a < op->d && rc == FKSKI_OK; ++a) {
        RealPass p;
        int64_t S = 1;
        for (int k = a + 1; k < op->d; ++k) S *= op->g.M[k];
        p.S = S;
        p.M = (int)op->g.M[a];
        p.L = op->L[a];
        p.lpr = m / p.M;
        p.lpr2 = p.lpr + (p.lpr & 1);
        p.nlines = (int64_t)nrhs * p.lpr2;
        p.Q = 2;
        rc = tune_pass<T>(op->dtype, p, (const T *)op->lam[a], (const typename Cx<T>::t *)op->tw[a], buf,
                          buf + (size_t)nrhs * m, s);
    }
    cudaFreeAsync(buf, s);
    return rc;
}

int kgop_tune(KgOp *op, int nrhs, cudaStream_t s) {
    if (op->kind != FKSKI_RBF || nrhs < 1) return FKSKI_OK;
    for (int a = 0; a < op->d; ++a)
        if (!op->lam[a] || !op->tw[a]) return FKSKI_E_INVALID_ARG;  // spectra first (kgop_set)
    if (op->dtype == FKSKI_F32) return kron_tune<float>(op, nrhs, s);
    if (op->dtype == FK_DF) return kron_tune<dfl>(op, nrhs, s);
    return kron_tune<double>(op, nrhs, s);
}

// One line per tuned pass shape: "dtype L M S lines -> radix cl threads ms".
size_t kg_tuning_table(char *buf, size_t len) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::string out;
    char line[200];
    for (const auto &kv : g_tune) {
        snprintf(line, sizeof(line), "%s L=%d M=%d S=%lld lines=%lld -> radix %d, %d lines/CTA, %d threads, %.4f ms\n",
                 kv.first.dtype == FKSKI_F32 ? "f32" : (kv.first.dtype == FK_DF ? "df" : "f64"), kv.first.L, kv.first.M, (long long)kv.first.S,
                 (long long)kv.first.nlines, kv.second.radix, kv.second.cl, kv.second.threads, (double)kv.second.ms);
        out += line;
    }
    if (buf && len > 0) {
        const size_t n = std::min(len - 1, out.size());
        memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return out.size() + 1;
}

template <typename T>
static int kron_apply(KgOp *op, const T *v, T *out, int nrhs, const T *addv, const double *alpha_dev, double alpha,
                      cudaStream_t s) {
    const int d = op->d;
    const int64_t m = op->m;
    if (d > 1) {
        FK_TRY(ensure(&op->scratch, op->scratch_bytes, sizeof(T) * (size_t)nrhs * m));
    }
    T *scr = (T *)op->scratch;
    // pass order: last axis first; buffers so that the final pass writes `out`
    const T *src = v;
    for (int step = 0; step < d; ++step) {
        const int a = d - 1 - step;
        T *dst;
        if (step == d - 1) dst = out;
        else dst = ((d - 1 - step) % 2 == 1) ? scr : out;
        RealPass p;
        int64_t S = 1;
        for (int k = a + 1; k < d; ++k) S *= op->g.M[k];
        p.S = S;
        p.M = (int)op->g.M[a];
        p.L = op->L[a];
        p.lpr = m / p.M;
        p.lpr2 = p.lpr + (p.lpr & 1);
        p.nlines = (int64_t)nrhs * p.lpr2;
        const PassCfg cfg = pass_config(op->dtype, p, nrhs);
        p.Q = 2 * cfg.cl;
        const bool last = step == d - 1;
        FK_TRY((launch_kron<T>(src, dst, p, cfg, (const T *)op->lam[a], (const typename Cx<T>::t *)op->tw[a],
                               last ? addv : nullptr, alpha_dev, alpha,
                               op->gate, s)));
        src = dst;
    }
    return FKSKI_OK;
}

template <typename T>
static int bttb_apply(KgOp *op, const T *v, T *out, int nrhs, const T *addv, const double *alpha_dev, double alpha,
                      cudaStream_t s) {
    using C = typename Cx<T>::t;
    const int d = op->d;
    const int64_t m = op->m;
    const int npair = nrhs;  // complex tensors, one per rhs
    // largest intermediate: M_0 x L_1 x ... x L_{d-1} complex per pair (or m complex)
    int64_t big = op->g.M[0];
    for (int k = 1; k < d; ++k) big *= op->L[k];
    big = std::max(big, m);
    FK_TRY(ensure(&op->scratch, op->scratch_bytes, 2 * sizeof(C) * (size_t)npair * big));
    C *z0 = (C *)op->scratch;
    C *z1 = z0 + (size_t)npair * big;
    const unsigned nb = (unsigned)std::min<int64_t>(cdiv((int64_t)npair * m, 256), 4096);
    k_pack_pairs<T><<<nb, 256, 0, s>>>(v, z0, m, nrhs, op->gate);
    FK_LAUNCH();
    int64_t ext[3] = {op->g.M[0], op->g.M[1], op->g.M[2]};
    C *cur = z0, *nxt = z1;
    // forward along axes d-1..1 (extent M -> L)
    for (int a = d - 1; a >= 1; --a) {
        CplxPass p = cplx_geom(ext, d, a, (int)op->g.M[a], op->L[a], op->L[a], npair);
        FK_TRY(launch_cplx<T>(cur, nxt, p, 0, (const T *)nullptr, s, op->gate));
        ext[a] = op->L[a];
        std::swap(cur, nxt);
    }
    // axis 0: forward, spectrum, inverse (extent M_0 -> M_0); spectrum lines indexed (k, rest)
    {
        CplxPass p = cplx_geom(ext, d, 0, (int)op->g.M[0], (int)op->g.M[0], op->L[0], npair);
        // lam is indexed [k * S + s] with S = prod_{k>0} L_k = p.S (the pair index folds into O)
        FK_TRY(launch_cplx<T>(cur, nxt, p, 2, (const T *)op->lamN, s, op->gate));
        std::swap(cur, nxt);
    }
    for (int a = 1; a < d; ++a) {
        CplxPass p = cplx_geom(ext, d, a, op->L[a], (int)op->g.M[a], op->L[a], npair);
        FK_TRY(launch_cplx<T>(cur, nxt, p, 1, (const T *)nullptr, s, op->gate));
        ext[a] = op->g.M[a];
        std::swap(cur, nxt);
    }
    const unsigned nb2 = (unsigned)std::min<int64_t>(cdiv((int64_t)nrhs * m, 256), 4096);
    k_unpack_pairs<T><<<nb2, 256, 0, s>>>(cur, out, m, nrhs, addv, alpha_dev, alpha, op->gate);
    FK_LAUNCH();
    return FKSKI_OK;
}

static int kgop_apply_any(KgOp *op, const void *v, void *out, int nrhs, const void *addv, const double *alpha_dev,
                          double alpha, cudaStream_t s) {
    if (op->kind < 0) return FKSKI_E_INVALID_ARG;
    if (nrhs < 1) return FKSKI_E_INVALID_ARG;
    if (op->kind == FKSKI_RBF) {
        if (op->dtype == FKSKI_F32)
            return kron_apply<float>(op, (const float *)v, (float *)out, nrhs, (const float *)addv, alpha_dev, alpha, s);
        if (op->dtype == FK_DF)
            return kron_apply<dfl>(op, (const dfl *)v, (dfl *)out, nrhs, (const dfl *)addv, alpha_dev, alpha, s);
        return kron_apply<double>(op, (const double *)v, (double *)out, nrhs, (const double *)addv, alpha_dev, alpha, s);
    }
    if (op->dtype == FKSKI_F32)
        return bttb_apply<float>(op, (const float *)v, (float *)out, nrhs, (const float *)addv, alpha_dev, alpha, s);
    if (op->dtype == FK_DF)
        return bttb_apply<dfl>(op, (const dfl *)v, (dfl *)out, nrhs, (const dfl *)addv, alpha_dev, alpha, s);
    return bttb_apply<double>(op, (const double *)v, (double *)out, nrhs, (const double *)addv, alpha_dev, alpha, s);
}

// Allocate the scratch an application to nrhs vectors needs (so graph capture allocates nothing).
int kgop_reserve(KgOp *op, int nrhs) {
    const size_t es = esz(op->dtype);
    const int d = op->d;
    size_t want = 0;
    if (op->kind == FKSKI_RBF) {
        if (d > 1) want = es * (size_t)nrhs * op->m;
    } else {
        int64_t big = op->g.M[0];
        for (int k = 1; k < d; ++k) big *= op->L[k];
        big = std::max(big, op->m);
        want = 2 * 2 * es * (size_t)nrhs * big;
    }
    if (want == 0) return FKSKI_OK;
    return ensure(&op->scratch, op->scratch_bytes, want);
}

void kgop_set_gate(KgOp *op, const int *gate) { op->gate = gate; }

int kgop_apply(KgOp *op, const void *v, void *out, int nrhs, const void *addv, double alpha, cudaStream_t s) {
    return kgop_apply_any(op, v, out, nrhs, addv, nullptr, alpha, s);
}

int kgop_apply_dev(KgOp *op, const void *v, void *out, int nrhs, const void *addv, const double *alpha_dev,
                   cudaStream_t s) {
    return kgop_apply_any(op, v, out, nrhs, addv, alpha_dev, 0.0, s);
}

int kg_mvm_impl(const fkski_grid *grid, const fkski_kernel *kern, int param, const void *v, void *out, int nrhs,
                int dtype, cudaStream_t s) {
    if (!grid || !kern || !v || !out || nrhs < 1) return FKSKI_E_INVALID_ARG;
    if (grid->d < 1 || grid->d > 3) return FKSKI_E_INVALID_ARG;
    if (dtype != FKSKI_F32 && dtype != FKSKI_F64 && dtype != FK_DF) return FKSKI_E_INVALID_ARG;
    for (int k = 0; k < grid->d; ++k)
        if (grid->M[k] < 4 || !(grid->h[k] > 0.0)) return FKSKI_E_INVALID_ARG;
    if (v == out) return FKSKI_E_INVALID_ARG;
    KgOp *op = nullptr;
    FK_TRY(kgop_create(grid, dtype, &op));
    int rc = kgop_set(op, kern, param, s);
    if (rc == FKSKI_OK) rc = kgop_apply(op, v, out, nrhs, nullptr, 0.0, s);
    cudaStreamSynchronize(s);  // op buffers are freed below
    kgop_destroy(op);
    return rc;
}

// ------------------------------------------------------------------ allocation-free K_G product
// For callers that may not allocate device memory at call time: code running while a
// cudaMalloc-free region is required (an allocator owned by someone else, a fixed memory
// budget checked up front, a host thread that must not take the allocator's locks).  The RBF
// Kronecker product needs only the d axis spectra and one intermediate of nrhs * m values, so
// both live in one fixed device array instead of buffers obtained per call.  That array is
// shared by every call on a device and keeps whatever the last call wrote: each call rewrites
// the spectra and the intermediate before reading them, so nothing in it has to start at zero,
// but two calls in flight at once on the same device (two streams, two host threads) overwrite
// each other's data and give wrong results.
static __device__ __align__(256) unsigned char g_kg_noalloc_scratch[FKSKI_NOALLOC_SCRATCH_BYTES];

constexpr size_t NOALLOC_LAM_BYTES = sizeof(double) * FFT_SMEM_CPLX;  // one axis spectrum (or twiddle table), FP32 or FP64
constexpr size_t NOALLOC_BUF_OFFSET = 6 * NOALLOC_LAM_BYTES;              // 3 spectra, 3 twiddle tables
constexpr int NOALLOC_MAX_DEVICES = 64;
static_assert(NOALLOC_BUF_OFFSET % 256 == 0, "intermediate must stay 256-byte aligned");
static_assert(FKSKI_NOALLOC_SCRATCH_BYTES > NOALLOC_BUF_OFFSET, "scratch smaller than its spectra");

static std::mutex g_noalloc_mu;
static void *g_noalloc_base[NOALLOC_MAX_DEVICES];

// Device address of the scratch array for the current device, looked up once per device.
static int noalloc_scratch(void **base) {
    int dev = -1;
    FK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return FKSKI_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        FK_CUDA(cudaGetSymbolAddress(&p, g_kg_noalloc_scratch));
        g_noalloc_base[dev] = p;
    }
    *base = g_noalloc_base[dev];
    return FKSKI_OK;
}

static size_t kg_noalloc_max_values(int dtype) {
    return (FKSKI_NOALLOC_SCRATCH_BYTES - NOALLOC_BUF_OFFSET) / esz(dtype);
}

int kg_mvm_noalloc_impl(const fkski_grid *grid, const fkski_kernel *kern, int param, const void *v, void *out,
                        int nrhs, int dtype, cudaStream_t s) {
    if (!grid || !kern || !v || !out || nrhs < 1) return FKSKI_E_INVALID_ARG;
    if (grid->d < 1 || grid->d > 3) return FKSKI_E_INVALID_ARG;
    if (dtype != FKSKI_F32 && dtype != FKSKI_F64) return FKSKI_E_INVALID_ARG;
    for (int k = 0; k < grid->d; ++k)
        if (grid->M[k] < 4 || !(grid->h[k] > 0.0)) return FKSKI_E_INVALID_ARG;
    if (v == out) return FKSKI_E_INVALID_ARG;
    if (kern->type != FKSKI_RBF) return FKSKI_E_UNSUPPORTED;
    KgOp op;
    memset(&op, 0, sizeof(op));
    op.g = *grid;
    op.d = grid->d;
    op.dtype = dtype;
    op.m = 1;
    op.N = 1;
    op.kind = -1;
    for (int a = 0; a < op.d; ++a) {
        op.m *= grid->M[a];
        op.L[a] = next_pow2(2 * grid->M[a] - 1);
        if (op.L[a] > FFT_SMEM_CPLX) return FKSKI_E_UNSUPPORTED;
        op.N *= op.L[a];
    }
    // the intermediate holds nrhs * m values (none for d = 1)
    if (op.d > 1 && (uint64_t)nrhs * (uint64_t)op.m > kg_noalloc_max_values(dtype)) return FKSKI_E_UNSUPPORTED;
    void *base = nullptr;
    FK_TRY(noalloc_scratch(&base));
    unsigned char *b = static_cast<unsigned char *>(base);
    for (int a = 0; a < op.d; ++a) {
        op.lam[a] = b + (size_t)a * NOALLOC_LAM_BYTES;
        op.tw[a] = b + (size_t)(3 + a) * NOALLOC_LAM_BYTES;
    }
    op.scratch = b + NOALLOC_BUF_OFFSET;
    op.scratch_bytes = FKSKI_NOALLOC_SCRATCH_BYTES - NOALLOC_BUF_OFFSET;
    // with the spectra, twiddles and the intermediate already in place, neither step below allocates
    FK_TRY(kgop_set(&op, kern, param, s));
    return kgop_apply(&op, v, out, nrhs, nullptr, 0.0, s);
}

}  // namespace fk
