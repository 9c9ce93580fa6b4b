// Definition of the opaque fcas_ctx, shared by the translation units that implement the C ABI.
#pragma once

#include <vector>

#include "fcas_ff.cuh"
#include "fcas_kernels.cuh"

namespace fcas {

// Record `msg` as the calling thread's last error (returned by fcas_last_error) and return `code`.
int report_error(int code, const char* msg);

struct EventPair {
    cudaEvent_t a, b;
    int kind;
};

// Bytes of the intermediate transform per particle: two series of N complex values.
inline size_t inter_bytes_per_particle(int precision, int64_t n_fft) {
    return (precision == FCAS_PREC_FP32 ? sizeof(float2) : sizeof(double2)) * (size_t)kSeries * (size_t)n_fft;
}

}  // namespace fcas

struct fcas_ctx {
    fcas_setup setup{};
    int device = -1;                // CUDA device current at create: every array of the context lives there
    int log_n = 0, log_n1 = 0, log_n2 = 0;
    int64_t n1 = 0, n2 = 0;
    int64_t k_lo = 0, k_hi = 0;
    double df = 0.0, scale = 1.0;
    double sigma2[FCAS_MAX_DET] = {};
    double* d_det = nullptr;        // [D][9]
    double* d_sigma2s = nullptr;    // scaled template norms
    double2* d_ynat = nullptr;      // whitened band spectrum in natural order [D][N/2] (binary64)
    int split_bias = 0;             // N2 = 2^(floor(log2 N / 2) - split_bias)
    int k1b = 0;                    // pass-A columns per CTA (layout of d_y and d_basis)
    int radix_bits_a = 4;           // pass-A full-stage radix bits (4: radix 16, 3: radix 8)
    int sub = 8;                    // pass-A column blocks scheduled together
    double tuned_ms = 0.0;          // per-particle time of the tuned configuration (0: not tuned)
    int64_t nb_cap = 0;             // argmax partials per particle the scratch holds
    void* d_y = nullptr;            // Y (precision-dependent)
    void* d_basis = nullptr;
    void* d_tw = nullptr;           // precision-dependent copies of the twiddle tables
    void* d_twlo = nullptr;
    void* d_twhi = nullptr;
    double2* d_tw64 = nullptr;      // binary64 tables (create path)
    double2* d_twlo64 = nullptr;
    double2* d_twhi64 = nullptr;
    float2* d_tw32 = nullptr;
    float2* d_twlo32 = nullptr;
    float2* d_twhi32 = nullptr;
    double2* d_stw_a64 = nullptr;   // per-stage twiddles, length-N2 transforms
    float2* d_stw_a32 = nullptr;
    double2* d_stw_b64 = nullptr;   // per-stage twiddles, length-N1 transforms
    float2* d_stw_b32 = nullptr;
    void* d_twloff = nullptr;       // float-float copies (16-byte entries) of twlo, twhi and the
    void* d_twhiff = nullptr;       // stage tables (FCAS_PREC_FF contexts only)
    void* d_stw_aff = nullptr;
    void* d_stw_bff = nullptr;
    void* d_phff = nullptr;         // float-float phasor table e^{2 pi i m / 1024} (FCAS_PREC_FF contexts only)
    fcas::ParticleParams* d_params = nullptr;
    int64_t params_cap = 0;
    double* d_theta = nullptr;      // staging for host theta
    double* d_fit = nullptr;        // staging for host outputs
    int64_t* d_tc = nullptr;
    int64_t stage_cap = 0;
    void* d_inter = nullptr;        // [chunk][2][N2][N1] complex
    fcas::Partial* d_partials = nullptr;  // [chunk][blocks per particle]
    int64_t chunk = 0;
    int64_t nb_partials = 0;
    // adjoint
    double* d_gsums = nullptr;       // [n][D][12] per-detector sums at t*
    double* d_gstage = nullptr;      // [n][4] gradient staging for host outputs
    int64_t grad_cap = 0;
    unsigned char* d_polish = nullptr;  // working arrays of fcas_polish
    size_t polish_bytes = 0;
    // particle swarm search
    unsigned char* d_pso = nullptr;  // state, parameters, fitness, counters and results of the swarm
    size_t pso_bytes = 0;
    cudaStream_t search_stream = nullptr;
    // profiling
    bool prof = false;
    std::vector<fcas::EventPair> events;
    size_t events_used = 0;
};

namespace fcas {

// FCAS_OK when the device current on the calling thread is the one the context was created on;
// otherwise FCAS_ERR_INVALID (or FCAS_ERR_CUDA) with a message naming `fn` and both devices.
int check_ctx_device(const fcas_ctx* c, const char* fn);
// FCAS_OK when p is memory the current device can use as device memory (device or managed
// allocation of that device); FCAS_ERR_INVALID with a message naming `fn` and `what` otherwise.
int check_device_array(const void* p, const char* fn, const char* what);

// Pointers and sizes the fitness kernels need, taken from a prepared context.
// Pass A / pass B of one chunk in the context's form.
inline cudaError_t launch_pass_a_prec(int precision, const FitnessPlan& plan, const ParticleParams* params, int64_t p0,
                                      int64_t np, void* inter, cudaStream_t st) {
    if (precision == FCAS_PREC_FP32) return launch_pass_a<float>(plan, params, p0, np, inter, st);
    if (precision == FCAS_PREC_FF) return launch_pass_a<ffloat>(plan, params, p0, np, inter, st);
    return launch_pass_a<double>(plan, params, p0, np, inter, st);
}
inline cudaError_t launch_pass_b_prec(int precision, const FitnessPlan& plan, const ParticleParams* params, int64_t p0,
                                      int64_t np, const void* inter, Partial* partials, cudaStream_t st) {
    if (precision == FCAS_PREC_FP32) return launch_pass_b<float>(plan, params, p0, np, inter, partials, st);
    if (precision == FCAS_PREC_FF) return launch_pass_b<ffloat>(plan, params, p0, np, inter, partials, st);
    return launch_pass_b<double>(plan, params, p0, np, inter, partials, st);
}

// bin step between a pass-A thread's consecutive values: N1 N2 / V_A, V_A = 2^min(log N2, radix bits)
inline int64_t pass_a_kstep(const fcas_ctx* c) {
    const int vb = c->log_n2 < c->radix_bits_a ? c->log_n2 : c->radix_bits_a;
    return (int64_t)1 << (c->log_n - vb);
}

inline FitnessPlan make_plan(const fcas_ctx* c) {
    FitnessPlan p;
    p.n_det = c->setup.n_det;
    p.log_n = c->log_n;
    p.log_n1 = c->log_n1;
    p.log_n2 = c->log_n2;
    p.n_samples = c->setup.n_samples;
    const bool fp32 = c->setup.precision == FCAS_PREC_FP32, ff = c->setup.precision == FCAS_PREC_FF;
    p.y = c->d_y;
    p.basis = c->d_basis;
    p.stw_a = fp32 ? (const void*)c->d_stw_a32 : ff ? (const void*)c->d_stw_aff : (const void*)c->d_stw_a64;
    p.stw_b = fp32 ? (const void*)c->d_stw_b32 : ff ? (const void*)c->d_stw_bff : (const void*)c->d_stw_b64;
    p.k1b = c->k1b;
    p.radix_bits_a = c->radix_bits_a;
    p.sub = c->sub;
    p.tw_lo = ff ? c->d_twloff : c->d_twlo;
    p.tw_hi = ff ? c->d_twhiff : c->d_twhi;
    p.ptab = c->d_phff;
    return p;
}

}  // namespace fcas
