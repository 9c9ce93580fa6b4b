// Double-word ("float-float") arithmetic for the FP32 units: a value is the unevaluated sum h + l
// of two floats with |l| <= ulp(h)/2 (Dekker 1971; error bounds of Joldes, Muller & Popescu 2017).
#pragma once

#include <cuda_runtime.h>

namespace fcas {

struct ffloat {
    float h, l;
    ffloat() = default;
    __host__ __device__ constexpr ffloat(float hi, float lo) : h(hi), l(lo) {}
    __host__ __device__ ffloat(double d) : h((float)d), l((float)(d - (double)(float)d)) {}
};

struct ff2 {
    ffloat x, y;
};

__host__ __device__ __forceinline__ double ff_to_double(ffloat a) { return (double)a.h + (double)a.l; }

#ifdef __CUDACC__
// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ float ff_two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ float ff_fast_two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
    return s;
}
// a + b with an absolute error of a few units of 2^-48 (|a| + |b|): enough for normwise-accurate
// transforms (the sloppy double-word sum: one two-sum of the high parts)
__device__ __forceinline__ ffloat ff_add(ffloat a, ffloat b) {
    float e;
    const float s = ff_two_sum(a.h, b.h, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    float lo;
    const float hi = ff_fast_two_sum(s, e, lo);
    return ffloat(hi, lo);
}
// a + b for a float b (the same sum with a zero low part of b)
__device__ __forceinline__ ffloat ff_add_f(ffloat a, float b) {
    float e;
    const float s = ff_two_sum(a.h, b, e);
    e = __fadd_rn(e, a.l);
    float lo;
    const float hi = ff_fast_two_sum(s, e, lo);
    return ffloat(hi, lo);
}
__device__ __forceinline__ ffloat ff_neg(ffloat a) { return ffloat(-a.h, -a.l); }
__device__ __forceinline__ ffloat ff_sub(ffloat a, ffloat b) { return ff_add(a, ff_neg(b)); }
// a b: the exact leading product by a fused multiply-add plus the cross terms (double-word product)
__device__ __forceinline__ ffloat ff_mul(ffloat a, ffloat b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    float lo;
    const float hi = ff_fast_two_sum(p, e, lo);
    return ffloat(hi, lo);
}

__device__ __forceinline__ ffloat operator+(ffloat a, ffloat b) { return ff_add(a, b); }
__device__ __forceinline__ ffloat operator-(ffloat a, ffloat b) { return ff_sub(a, b); }
__device__ __forceinline__ ffloat operator-(ffloat a) { return ff_neg(a); }
__device__ __forceinline__ ffloat operator*(ffloat a, ffloat b) { return ff_mul(a, b); }
__device__ __forceinline__ ffloat& operator+=(ffloat& a, ffloat b) { return a = ff_add(a, b); }
__device__ __forceinline__ bool operator>(ffloat a, ffloat b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }
__device__ __forceinline__ bool operator==(ffloat a, ffloat b) { return a.h == b.h && a.l == b.l; }

__device__ __forceinline__ ff2 operator+(ff2 a, ff2 b) { return ff2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ ff2 operator-(ff2 a, ff2 b) { return ff2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ ff2 cmul(ff2 a, ff2 b) { return ff2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ ff2 cconj(ff2 a) { return ff2{a.x, -a.y}; }
__device__ __forceinline__ ff2 mkc(ffloat x, ffloat y) { return ff2{x, y}; }
template <int S> __device__ __forceinline__ ff2 mul_si(ff2 a) { return S > 0 ? ff2{-a.y, a.x} : ff2{a.y, -a.x}; }

__device__ __forceinline__ float shfl_down_r(float v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }
__device__ __forceinline__ double shfl_down_r(double v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }
__device__ __forceinline__ ffloat shfl_down_r(ffloat v, int off) {
    return ffloat(__shfl_down_sync(0xffffffffu, v.h, off), __shfl_down_sync(0xffffffffu, v.l, off));
}
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(ffloat v) { return ff_to_double(v); }
#endif

}  // namespace fcas
