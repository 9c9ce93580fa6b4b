// Packed two-series FP32 arithmetic for the FP32 form of the fitness passes.
//
// Pass A produces, and pass B transforms, two network-weighted series per particle (W_1 and W_2,
// Sec. II.C projection taken before the t_c transform). Both go through identical transforms with
// identical twiddles, so one thread carries both: lane 0 of a packed 64-bit register holds the value
// of the first series and lane 1 that of the second, and one packed FP32 instruction (add, sub, mul
// or fma .f32x2, sm_100 and later) does the work of two scalar ones. A complex value of both series
// is c32x2 {x = (re_1, re_2), y = (im_1, im_2)}, 16 bytes, stored as (re_1, re_2, im_1, im_2) in
// shared and global memory so that one 16-byte access moves both series.
//
// Packed instructions take no immediate operands and no negated operands: multiplications by +-i
// are folded into the neighbouring additions by the transforms (add_si / sub_si), and constant
// rotations keep their negated constants in registers. Twiddles stay scalar (one float2 shared by
// both lanes): their products are formed once for both series and applied with scalar FP32
// instructions on the two halves of each packed register.
#pragma once

#include <cuda_runtime.h>


namespace fcas {

struct f32x2 {
    unsigned long long v;
};
struct __align__(16) c32x2 {
    f32x2 x, y;
};
// tag of the packed two-series form (cplx<x2f> is c32x2, its twiddles are float2)
struct x2f {};
template <typename R> struct cplx_of;
template <> struct cplx_of<x2f> { using type = c32x2; };

#ifdef __CUDACC__
__device__ __forceinline__ f32x2 pk2(float lane0, float lane1) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lane0), "f"(lane1));
    return r;
}
__device__ __forceinline__ float2 upk2(f32x2 a) {
    float l0, l1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l0), "=f"(l1) : "l"(a.v));
    return make_float2(l0, l1);
}
__device__ __forceinline__ f32x2 bcast2(float c) { return pk2(c, c); }

__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
// a b + c, one rounding per lane
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ f32x2 neg2(f32x2 a) { return bcast2(0.0f) - a; }

__device__ __forceinline__ c32x2 mkc(f32x2 x, f32x2 y) { return c32x2{x, y}; }
__device__ __forceinline__ c32x2 operator+(c32x2 a, c32x2 b) { return c32x2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ c32x2 operator-(c32x2 a, c32x2 b) { return c32x2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ c32x2 zero_c32x2() { return c32x2{bcast2(0.0f), bcast2(0.0f)}; }
// both series from their scalar values
__device__ __forceinline__ c32x2 pack_series(float2 s1, float2 s2) { return c32x2{pk2(s1.x, s2.x), pk2(s1.y, s2.y)}; }

// a w for a twiddle w shared by both series: scalar FP32 on the halves of the packed registers
// (the same operations per series as the scalar complex product)
__device__ __forceinline__ c32x2 cmul(c32x2 a, float2 w) {
    const float2 re = upk2(a.x), im = upk2(a.y);
    const float r0 = fmaf(re.x, w.x, -im.x * w.y), i0 = fmaf(re.x, w.y, im.x * w.x);
    const float r1 = fmaf(re.y, w.x, -im.y * w.y), i1 = fmaf(re.y, w.y, im.y * w.x);
    return c32x2{pk2(r0, r1), pk2(i0, i1)};
}

// x e^{S 2 pi i M / 16}, M in 0..15 (constant rotations of the radix-16 and radix-8 butterflies)
template <int S, int M>
__device__ __forceinline__ c32x2 rot16_x2(c32x2 x) {
    constexpr int m = M & 15;
    constexpr float kC8 = 0.92387953251128675613f, kS8 = 0.38268343236508977173f, kR2 = 0.70710678118654752440f;
    if constexpr (m == 0) {
        return x;
    } else if constexpr (m == 4 || m == 12) {
        // S' i x with S' = S (m = 4) or -S (m = 12): (-S' y, S' x)
        constexpr int sp = m == 4 ? S : -S;
        return sp > 0 ? c32x2{neg2(x.y), x.x} : c32x2{x.y, neg2(x.x)};
    } else if constexpr (m == 8) {
        return c32x2{neg2(x.x), neg2(x.y)};
    } else if constexpr ((m & 3) == 2) {
        // |cos| = |sin| = 1/sqrt 2: c = sc k, s = ss k
        constexpr int sc = (m == 2 || m == 14) ? 1 : -1;
        constexpr int ss = S * ((m == 2 || m == 6) ? 1 : -1);
        const f32x2 k = bcast2(sc > 0 ? kR2 : -kR2);
        if constexpr (sc == ss) return c32x2{(x.x - x.y) * k, (x.x + x.y) * k};
        else return c32x2{(x.x + x.y) * k, (x.y - x.x) * k};
    } else {
        // odd m: c = cos(2 pi m / 16), s = S sin(2 pi m / 16) from the first-octant pair
        constexpr float ca = (m == 1 || m == 15) ? kC8 : (m == 3 || m == 13) ? kS8 : (m == 5 || m == 11) ? -kS8 : -kC8;
        constexpr float sa = (m == 1 || m == 7) ? kS8 : (m == 3 || m == 5) ? kC8 : (m == 9 || m == 15) ? -kS8 : -kC8;
        constexpr float c = ca, s = S > 0 ? sa : -sa;
        const f32x2 vc = bcast2(c), vs = bcast2(s), vns = bcast2(-s);
        return c32x2{fma2(x.y, vns, x.x * vc), fma2(x.y, vc, x.x * vs)};
    }
}

// read-only load that does not allocate in L1 (pass B reads each intermediate element once)
__device__ __forceinline__ c32x2 ld_na(const c32x2* p) {
    c32x2 r;
    asm("ld.global.nc.L1::no_allocate.v2.b64 {%0, %1}, [%2];" : "=l"(r.x.v), "=l"(r.y.v) : "l"(p));
    return r;
}
// streamed store (evict-first): pass A's output is read back once, by pass B
__device__ __forceinline__ void st_stream_x2(c32x2* p, c32x2 v) {
    asm volatile("st.global.cs.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(v.x.v), "l"(v.y.v) : "memory");
}
// |W_1|^2 + |W_2|^2 of one element: both lanes' squared magnitudes, then their sum
__device__ __forceinline__ float norm2_sum(c32x2 a) {
    const float2 g = upk2(fma2(a.y, a.y, a.x * a.x));
    return g.x + g.y;
}
#endif

}  // namespace fcas
