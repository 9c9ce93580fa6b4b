// Kernel launchers of the fitness path (defined in fcas_kernels.cu) and of the create path
// (fcas_create.cu).
#pragma once

#include "fcas_internal.cuh"

namespace fcas {

// Chirp-phase basis of one bin for the FP32 form: phi^-1/3 as a float-float pair (hi, lo); the
// powers phi^-2/3, phi^-1, phi^-5/3 are formed from it by float-float products.
struct __align__(8) BasisF {
    float h, l;
};

// (ah + al)(bh + bl) as a float-float pair: the exact leading product by a fused multiply-add,
// the cross terms added to its error, then renormalised (double-word product, relative error a
// few units of 2^-48).
__host__ __device__ __forceinline__ float2 ff_mul(float ah, float al, float bh, float bl) {
#ifdef __CUDA_ARCH__
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float hi = __fadd_rn(p, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, p)));
#else
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float hi = p + e;
    return make_float2(hi, e - (hi - p));
#endif
}

// phi^-5/3, phi^-1, phi^-2/3, phi^-1/3 (hi, lo pairs) of a bin from its basis t = phi^-1/3
struct ChirpPowers {
    float2 b53, b1, b23, b13;
};
__host__ __device__ __forceinline__ ChirpPowers chirp_powers(const BasisF& t) {
    ChirpPowers r;
    r.b13 = make_float2(t.h, t.l);
    r.b23 = ff_mul(t.h, t.l, t.h, t.l);
    r.b1 = ff_mul(r.b23.x, r.b23.y, t.h, t.l);
    r.b53 = ff_mul(r.b1.x, r.b1.y, r.b23.x, r.b23.y);
    return r;
}
#ifdef __CUDACC__
// The same powers as unnormalised pairs (p, e): the exact leading product plus the cross terms,
// |e| within a few ulp(p). Renormalising only moves bits between the two words, so the pairs carry
// the same value to the same accuracy (a few units of 2^-46 relative) for the products and phase
// fractions that take them next, three instructions fewer per product.
__device__ __forceinline__ float2 ff_mul_raw(float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    return make_float2(p, e);
}
// frac((ah + al)(bh + bl)) with the leading product split exactly: the result is the product
// reduced by an integer, accurate to a few float ulps of 1 turn (the FP32 form's phase fractions).
__device__ __forceinline__ float frac_mul_ff(float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    return __fadd_rn(__fsub_rn(p, rintf(p)), e);
}
__device__ __forceinline__ ChirpPowers chirp_powers_lean(const BasisF& t) {
    ChirpPowers r;
    r.b13 = make_float2(t.h, t.l);
    r.b23 = ff_mul_raw(t.h, t.l, t.h, t.l);
    r.b1 = ff_mul_raw(r.b23.x, r.b23.y, t.h, t.l);
    r.b53 = ff_mul_raw(r.b1.x, r.b1.y, r.b23.x, r.b23.y);
    return r;
}
#endif
struct __align__(16) BasisD {
    double2 a;  // (b53, b1)
    double2 b;  // (b23, b13)
};
template <typename R> struct basis_of;
template <> struct basis_of<float> { using type = BasisF; };
template <> struct basis_of<double> { using type = BasisD; };
template <typename R> using Basis = typename basis_of<R>::type;

struct Partial {
    double val;
    int64_t t;
};

struct FitnessPlan {
    int n_det;
    int log_n, log_n1, log_n2;
    int64_t n_samples;
    const void* y;                // Y layout [k1 / K1B][i][k2 < N2/2][k1 % K1B]
    const void* basis;            // basis layout [k1 / K1B][k2 < N2/2][k1 % K1B]
    const void* stw_a;            // per-stage twiddles of the length-N2 transforms
    const void* stw_b;            // per-stage twiddles of the length-N1 transforms
    int k1b;                      // columns per pass-A CTA (must match the layout of y and basis)
    int radix_bits_a;             // pass-A full-stage radix bits (4: radix 16, 3: radix 8; matches stw_a)
    int sub;                      // adjacent column blocks of a particle scheduled together
    const void* tw_lo;            // e^{2 pi i m / N}, m < 4096
    const void* tw_hi;            // e^{2 pi i 4096 m / N}, m < max(1, N / 4096)
    const void* ptab;             // float-float e^{2 pi i m / 1024}, m < 1024 (FCAS_PREC_FF only)
};

// Per-particle geometry (binary64): chirp coefficients, delays, antenna patterns, G^-1.
// kstep: the bin step between a pass-A thread's consecutive values (N / V_A, pass_a_kstep).
cudaError_t launch_geometry(const double* theta, int64_t n, ParticleParams* out, const double* det9,
                            const double* sigma2_scaled, int n_det, double f_star, double df, int64_t kstep,
                            cudaStream_t s);

// Pass A for particles [p0, p0 + np): writes the intermediate [np][2][N2][N1].
template <typename Real>
cudaError_t launch_pass_a(const FitnessPlan& plan, const ParticleParams* params, int64_t p0, int64_t np,
                          void* inter, cudaStream_t s);
// Pass B + projection + partial argmax: writes partials [np][N2 / TB].
template <typename Real>
cudaError_t launch_pass_b(const FitnessPlan& plan, const ParticleParams* params, int64_t p0, int64_t np,
                          const void* inter, Partial* partials, cudaStream_t s);
// Final argmax: fitness[p0 + p], tc[p0 + p].
cudaError_t launch_reduce(const Partial* partials, int64_t nb, const ParticleParams* params, int64_t p0,
                          int64_t np, double* fitness, int64_t* tc, cudaStream_t s);

int pass_b_blocks_per_particle(int log_n1, int log_n2, int precision);
// Checked build (FCAS_CHECKED): waits for the stream, returns and clears the bits of the index
// checks that failed since the last call (see fcas_fft16.cuh). Other builds: 0, no synchronisation.
unsigned int take_index_checks(cudaStream_t s);
// float-float copy (16-byte entries: hi/lo of re, hi/lo of im) of a binary64 complex table
cudaError_t launch_split_ff(const double2* src, void* dst, int64_t n, cudaStream_t s);
// float-float table of e^{2 pi i m / n}, m < n (16-byte entries as above)
cudaError_t launch_phase_table_ff(void* dst, int n, cudaStream_t s);
unsigned int take_index_checks_ff(cudaStream_t s);   // the float-float passes' translation unit
int pass_a_k1b_for(int log_n2, int precision);
// compiled pass-A column-block widths (radix-16 stages) for a length: writes up to 4 values, returns the count
int pass_a_k1b_variants(int log_n2, int precision, int* out);
cudaError_t launch_stage_tables(int log_l, int maxrb, double2* t64, float2* t32, cudaStream_t s);
// pass A with radix-8 stages (8 values per thread) is compiled for these shapes
bool pass_a_radix8_available(int log_n2, int precision, int k1b);
// pass-A stage radix bits a context starts with (and fcas_set_shape's radix_bits_a = 0)
int pass_a_default_radix_bits(int log_n2, int precision);

// ---- adjoint (fcas_grad.cu) ----
template <typename Real>
cudaError_t launch_grad_sums(const FitnessPlan& pl, int k1b, int64_t k_lo, int64_t k_hi, const ParticleParams* params,
                             const int64_t* tc, int64_t n, double* sums, cudaStream_t s, bool y_ff = false);
cudaError_t launch_grad_final(const double* theta, const int64_t* tc, int64_t n, const double* sums,
                              const double* det9, const double* s2, int n_det, double f_star, double df, double* grad,
                              cudaStream_t s);

// ---- gradient polishing (fcas_grad.cu) ----
struct PolishScales {
    double s[4];   // step scales: absolute for alpha, delta; relative (times tau0, tau1.5) for the chirp times
};
cudaError_t launch_polish_direction(const double* theta, const double* grad, const PolishScales& sc, int64_t n,
                                    double* dir, double* step, int32_t* done, cudaStream_t s);
cudaError_t launch_polish_candidate(const double* theta, const double* dir, const double* step, const int32_t* done,
                                    int64_t n, double* cand, cudaStream_t s);
cudaError_t launch_polish_accept(double* theta, double* fit, int64_t* tc, const double* cand, const double* cfit,
                                 const int64_t* ctc, double* step, int32_t* done, int32_t* accepted, int64_t n,
                                 int32_t* searching, cudaStream_t s);

// ---- create path (fcas_create.cu) ----
cudaError_t launch_tables(int log_n, int log_n1, int log_n2, double2* tw64, double2* twlo64, double2* twhi64,
                          float2* tw32, float2* twlo32, float2* twhi32, cudaStream_t s);
cudaError_t launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t s);
struct DetShifts {
    int64_t s[FCAS_MAX_DET];   // circular shift of each detector's series, 0..n_samples-1
};
cudaError_t launch_time_shift(const double* x, double* y, int n_det, int64_t n, const DetShifts& sh, cudaStream_t s);
cudaError_t launch_check_psd(const double* psd, int n_det, int64_t row, int64_t k_lo, int64_t k_hi, int* flag,
                             cudaStream_t s);
// the analytic aLIGO fit on the band bins of every detector's row (fcas_create with psd = NULL)
cudaError_t launch_analytic_psd(double* psd, int n_det, int64_t row, int64_t k_lo, int64_t k_hi, double df,
                                cudaStream_t s);
cudaError_t launch_sigma2(const double* psd, int n_det, int64_t row, int64_t k_lo, int64_t k_hi, double df,
                          double* sigma2, double* work, cudaStream_t s);
cudaError_t launch_data_fft(const double* data, int n_det, int64_t n_samples, int log_n, int log_n1, int log_n2,
                            const double2* tw64, int tw_shift_a, int tw_shift_b, const double2* twlo64,
                            const double2* twhi64, double2* work, double2* spec, cudaStream_t s);
cudaError_t launch_whiten(const double2* spec, const double* psd, int n_det, int64_t psd_row, int log_n, int64_t k_lo,
                          int64_t k_hi, double fs, double scale, double2* ynat, cudaStream_t s);
cudaError_t launch_layout(const double2* ynat, int n_det, int log_n, int log_n1, int log_n2, int k1b, int64_t k_lo,
                          int64_t k_hi, double fs, double f_star, int precision, void* y, void* basis, cudaStream_t s);

}  // namespace fcas
