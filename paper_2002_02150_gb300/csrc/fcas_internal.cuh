// Internal declarations shared by the CUDA translation units of libfcas.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fcas.h"

namespace fcas {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kCLight = 299792458.0;
constexpr double kRank1Rtol = 1e-12;   // det G < kRank1Rtol (tr G / 2)^2 -> rank-1 projection
constexpr int kTwLoBits = 12;          // two-level table for e^{2 pi i m / N}: m = hi * 4096 + lo

// ------------------------------------------------------------------------------------------
// complex helpers on float2 / double2
// ------------------------------------------------------------------------------------------
template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename R> using cplx = typename cplx_of<R>::type;

__host__ __device__ __forceinline__ float2 mkc(float x, float y) { return make_float2(x, y); }
__host__ __device__ __forceinline__ double2 mkc(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// multiply by S*i (S = +1 or -1)
template <int S> __device__ __forceinline__ float2 mul_si(float2 a) {
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <int S> __device__ __forceinline__ double2 mul_si(double2 a) {
    return S > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// ------------------------------------------------------------------------------------------
// Per-particle quantities computed once per evaluation in binary64 (geometry kernel).
// ------------------------------------------------------------------------------------------
struct ParticleParams {
    double c[4];                   // chirp phase coefficients [turns] of phi^-5/3, phi^-1, phi^-2/3, phi^-1/3
    double dturn[FCAS_MAX_DET];    // Delta^i * df: delay phase [turns] per frequency bin
    double u[FCAS_MAX_DET][2];     // U^i = (F+, Fx)(alpha, delta, psi = 0)
    double ginv[3];                // (G^-1)_{11}, (G^-1)_{12}, (G^-1)_{22} with the scaled template norms
    double chol[3];                // G^-1 = L L^T, L = [[l11, 0], [l21, l22]]: (l11, l21, l22)
    // Network weights: Gamma^2(t) = |sum_i w1_i Z_i(t)|^2 + |sum_i w2_i Z_i(t)|^2 with
    // w1_i = l11 U+^i + l21 Ux^i, w2_i = l22 Ux^i (L^T applied to U).
    double w1[FCAS_MAX_DET], w2[FCAS_MAX_DET];
    // float-float copies for the FP32 form (hi + lo)
    float ch[4], cl[4];
    float dh[FCAS_MAX_DET], dl[FCAS_MAX_DET];
    float w1f[FCAS_MAX_DET], w2f[FCAS_MAX_DET];
    float2 dstep[FCAS_MAX_DET];    // e^{2 pi i S Delta^i df}, S = N / V_A: the FP32 pass A's step of the
                                   // delay phasor between a thread's consecutive bins (binary64 phase)
    int32_t valid;                 // 0: non-finite / non-positive input -> fitness NaN, tc -1
    int32_t taylor_ok;             // FP32 pass A may step the chirp phase from an anchor bin to the
                                   // next 3 (bit 0) or 7 (bit 1) bins: remainder below 1e-7 turns
};

// ------------------------------------------------------------------------------------------
// Launch shapes. Pass A transforms columns of length N2 (K1B columns per CTA), pass B rows of
// length N1 (TB rows per CTA); each transform is held by L / V threads with V = min(16, L)
// values per thread. Pass A also keeps K1B <= L so that K1B divides N1 (N1 >= N2 = L).
// ------------------------------------------------------------------------------------------
__host__ __device__ constexpr int imin_c(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int imax_c(int a, int b) { return a > b ? a : b; }
#ifndef FCAS_PASS_A_THREADS_F32
#define FCAS_PASS_A_THREADS_F32 512   // target CTA size of pass A, FP32 form
#endif
#ifndef FCAS_PASS_A_SUB
#define FCAS_PASS_A_SUB 8             // adjacent column blocks of one particle scheduled together
#endif
#ifndef FCAS_SPLIT_BIAS
#define FCAS_SPLIT_BIAS 0             // N2 = 2^(floor(log2 N / 2) - bias): a smaller pass-A transform
#endif
#ifndef FCAS_PASS_B_THREADS_F32
#define FCAS_PASS_B_THREADS_F32 256   // target CTA size of pass B, FP32 form
#endif
__host__ __device__ constexpr int shape_v(int log_l) { return log_l >= 4 ? 16 : (1 << log_l); }
__host__ __device__ constexpr int pass_a_k1b(int log_l, int real_bytes) {
    return imin_c(imin_c(16, imax_c(1, (real_bytes == 4 ? FCAS_PASS_A_THREADS_F32 : 256) /
                                           ((1 << log_l) / shape_v(log_l)))),
                  1 << log_l);
}
__host__ __device__ constexpr int pass_a_threads(int log_l, int real_bytes) {
    return pass_a_k1b(log_l, real_bytes) * ((1 << log_l) / shape_v(log_l));
}
__host__ __device__ constexpr int pass_b_tb(int log_l, int real_bytes) {
    return imin_c(imin_c(16, imax_c(1, (real_bytes == 4 ? FCAS_PASS_B_THREADS_F32 : 128) /
                                           ((1 << log_l) / shape_v(log_l)))),
                  (1 << log_l) / 2);
}
__host__ __device__ constexpr int pass_b_threads(int log_l, int real_bytes) {
    return pass_b_tb(log_l, real_bytes) * ((1 << log_l) / shape_v(log_l));
}
// Transforms per particle between the passes: the two network-weighted series.
constexpr int kSeries = 2;

// Smallest/largest supported transform lengths; each pass transforms at most 2^13 points.
constexpr int kMinLogN = 4;
constexpr int kMaxLogN = 24;
constexpr int kMaxLogPass = 13;
__host__ __device__ constexpr int split_log_n2_with(int log_n, int bias) {
    return imax_c(2, imax_c(log_n - kMaxLogPass, log_n / 2 - bias));
}

}  // namespace fcas
