// Double-float ("float-float") arithmetic for the MIXED solver: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits, computed on the
// FP32 pipes.  GB300's FP64 rate is a small fraction of its FP32 rate, and the factorized CG
// needs operator products accurate far beyond FP32 to keep the iteration counts of exact-
// arithmetic CG (App. C.2; a per-product relative error of 1e-7 doubles them on the test
// systems), so the bulk arithmetic of MIXED runs in this form instead of FP64.
//
// The building blocks are the classical error-free transformations:
//   TwoSum   (Knuth, TAOCP vol. 2, 4.2.2):  s = fl(a + b) and the exact error e, a + b = s + e;
//   Fast2Sum (Dekker 1971), valid when |a| >= |b| (or a = 0);
//   TwoProd  with a fused multiply-add:      p = fl(a b), e = fma(a, b, -p), a b = p + e exactly.
// The addition is Dekker's form (TwoSum of the high parts, low parts added, renormalised): its
// error is below about 2^-46 (|a| + |b|), i.e. normwise like FP64 arithmetic with a 46-bit
// mantissa.  Every rounding goes through an explicit round-to-nearest intrinsic so the compiler
// can neither contract nor reassociate it; results are deterministic.
#pragma once

#include <cuda_runtime.h>

namespace fk {

struct __align__(8) dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit constexpr dfl(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ explicit constexpr dfl(float v) : hi(v), lo(0.f) {}
    __host__ __device__ explicit dfl(double v) {
#ifdef __CUDA_ARCH__
        hi = __double2float_rn(v);
        lo = __double2float_rn(__dsub_rn(v, (double)hi));
#else
        hi = (float)v;
        lo = (float)(v - (double)hi);
#endif
    }
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

struct __align__(16) dfl2 {
    dfl x, y;
};

#ifdef __CUDA_ARCH__
__device__ __forceinline__ float df_add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float df_sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float df_mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float df_fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float df_add_rn(float a, float b) { volatile float r = a + b; return r; }
inline float df_sub_rn(float a, float b) { volatile float r = a - b; return r; }
inline float df_mul_rn(float a, float b) { volatile float r = a * b; return r; }
inline float df_fma_rn(float a, float b, float c) { return fmaf(a, b, c); }
#endif

// TwoSum: s + e = a + b exactly.
__host__ __device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = df_add_rn(a, b);
    const float bb = df_sub_rn(s, a);
    e = df_add_rn(df_sub_rn(a, df_sub_rn(s, bb)), df_sub_rn(b, bb));
    return s;
}

// Fast2Sum: s + e = a + b exactly when |a| >= |b|.
__host__ __device__ __forceinline__ float fast_two_sum(float a, float b, float &e) {
    const float s = df_add_rn(a, b);
    e = df_sub_rn(b, df_sub_rn(s, a));
    return s;
}

__host__ __device__ __forceinline__ dfl df_renorm(float s, float e) {
    float l;
    const float h = fast_two_sum(s, e, l);
    return dfl(h, l);
}

__host__ __device__ __forceinline__ dfl operator+(const dfl a, const dfl b) {
    float e;
    const float s = two_sum(a.hi, b.hi, e);
    e = df_add_rn(e, df_add_rn(a.lo, b.lo));
    return df_renorm(s, e);
}

__host__ __device__ __forceinline__ dfl operator-(const dfl a) { return dfl(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dfl operator-(const dfl a, const dfl b) { return a + (-b); }

__host__ __device__ __forceinline__ dfl operator*(const dfl a, const dfl b) {
    const float p = df_mul_rn(a.hi, b.hi);
    float e = df_fma_rn(a.hi, b.hi, -p);
    e = df_fma_rn(a.hi, b.lo, e);
    e = df_fma_rn(a.lo, b.hi, e);
    return df_renorm(p, e);
}

// a * b + c * d (the parts of a complex product) with one normalisation: the exact high products
// (TwoProd) meet in one TwoSum; their errors and the cross terms a.hi b.lo, a.lo b.hi, c.hi d.lo,
// c.lo d.hi go into one FP32 sum.  19 operations against 25 for two products and a sum.
__host__ __device__ __forceinline__ dfl df_dot2(const dfl a, const dfl b, const dfl c, const dfl d) {
    const float p = df_mul_rn(a.hi, b.hi);
    const float q = df_mul_rn(c.hi, d.hi);
    float e = df_fma_rn(a.hi, b.hi, -p);
    e = df_fma_rn(a.hi, b.lo, e);
    e = df_fma_rn(a.lo, b.hi, e);
    e = df_add_rn(e, df_fma_rn(c.hi, d.hi, -q));
    e = df_fma_rn(c.hi, d.lo, e);
    e = df_fma_rn(c.lo, d.hi, e);
    float t;
    const float s = two_sum(p, q, t);
    return df_renorm(s, df_add_rn(t, e));
}

// dfl times an FP32 number (band values, twiddles that are exact in FP32).
__host__ __device__ __forceinline__ dfl df_mul_f(const dfl a, const float b) {
    const float p = df_mul_rn(a.hi, b);
    float e = df_fma_rn(a.hi, b, -p);
    e = df_fma_rn(a.lo, b, e);
    return df_renorm(p, e);
}

__host__ __device__ __forceinline__ dfl &operator+=(dfl &a, const dfl b) { return a = a + b; }
__host__ __device__ __forceinline__ dfl &operator-=(dfl &a, const dfl b) { return a = a - b; }
__host__ __device__ __forceinline__ dfl &operator*=(dfl &a, const dfl b) { return a = a * b; }

// a * b + c (product and sum each as above).  The math library's fma overloads stay visible
// inside this namespace next to this one.
using ::fma;
__host__ __device__ __forceinline__ dfl fma(const dfl a, const dfl b, const dfl c) { return a * b + c; }

// Accumulate the FP32 product b * x (x a dfl) into acc: TwoProd of the high parts, the low part's
// product in FP32 (it is 2^-24 smaller), then the Dekker addition.
__host__ __device__ __forceinline__ void df_acc_fx(dfl &acc, const float b, const dfl x) {
    const float p = df_mul_rn(b, x.hi);
    float e = df_fma_rn(b, x.hi, -p);
    e = df_fma_rn(b, x.lo, e);
    float t;
    const float s = two_sum(acc.hi, p, t);
    t = df_add_rn(t, df_add_rn(acc.lo, e));
    acc = df_renorm(s, t);
}

// Long sums of FP32-times-double-float products (the band product: 343 terms per node).  The
// accumulator keeps the running FP32 sum s of the products' high parts and, apart, the FP32 sum c
// of everything TwoSum and TwoProd left over; it is normalised once, at the end.  Each term costs
// 11 operations, and the dependence from one term to the next is a single addition on s and one
// on c, so the per-node chains do not serialise the whole sum.  The leftovers are 2^-24 smaller
// than the terms, so their FP32 rounding contributes about 2^-48 per term relative to the sum of
// the terms' magnitudes.
struct dacc {
    float s, c;
};

__host__ __device__ __forceinline__ void dacc_zero(dacc &a) { a.s = 0.f; a.c = 0.f; }

__host__ __device__ __forceinline__ void dacc_add_fx(dacc &a, const float b, const dfl x) {
    const float p = df_mul_rn(b, x.hi);
    float e = df_fma_rn(b, x.hi, -p);
    e = df_fma_rn(b, x.lo, e);
    float t;
    a.s = two_sum(a.s, p, t);
    a.c = df_add_rn(a.c, df_add_rn(t, e));
}

__host__ __device__ __forceinline__ dfl dacc_value(const dacc a) { return df_renorm(a.s, a.c); }

__host__ __device__ __forceinline__ bool df_isfinite(const dfl a) { return isfinite(a.hi) && isfinite(a.lo); }

}  // namespace fk
