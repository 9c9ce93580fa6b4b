// C ABI of libfcas: context lifetime, input validation, memory management and the launch
// sequence of one fitness evaluation (geometry -> per chunk: pass A -> pass B -> reduce).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fcas_ctx.cuh"
#include "fcas_diag.cuh"
#include "fcas_kernels.cuh"
#include "fcas_pso.cuh"

using namespace fcas;

namespace {

// Host-side NVTX range around each C entry point (visible to ncu --nvtx and other NVTX tools;
// a no-op when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};


thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define FCAS_CUDA(call)                                                                              \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(FCAS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace fcas {
int report_error(int code, const char* msg) {
    g_last_error = msg;
    return code;
}

int check_ctx_device(const fcas_ctx* c, const char* fn) {
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(FCAS_ERR_CUDA, "%s: cudaGetDevice: %s", fn, cudaGetErrorString(e));
    if (dev != c->device)
        return fail(FCAS_ERR_INVALID, "%s: the context was created on device %d but device %d is current", fn,
                    c->device, dev);
    return FCAS_OK;
}

int check_device_array(const void* p, const char* fn, const char* what) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(FCAS_ERR_CUDA, "%s: cudaGetDevice: %s", fn, cudaGetErrorString(e));
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(FCAS_ERR_INVALID, "%s: %s is not a CUDA pointer", fn, what);
    }
    if (a.type == cudaMemoryTypeManaged) return FCAS_OK;
    if (a.type != cudaMemoryTypeDevice)
        return fail(FCAS_ERR_INVALID, "%s: %s must be device memory (host arrays would need staging memory)", fn, what);
    if (a.device != dev)
        return fail(FCAS_ERR_INVALID, "%s: %s lives on device %d but device %d is current", fn, what, a.device, dev);
    return FCAS_OK;
}
}  // namespace fcas

namespace {

void free_ctx(fcas_ctx* c) {
    void* ptrs[] = {c->d_det, c->d_sigma2s, c->d_y, c->d_basis, c->d_tw64, c->d_twlo64, c->d_twhi64,
                    c->d_tw32, c->d_twlo32, c->d_twhi32, c->d_stw_a64, c->d_stw_a32, c->d_stw_b64, c->d_stw_b32,
                    c->d_twloff, c->d_twhiff, c->d_stw_aff, c->d_stw_bff, c->d_phff,
                    c->d_params, c->d_theta, c->d_fit, c->d_tc, c->d_inter, c->d_partials, c->d_pso,
                    c->d_gsums, c->d_gstage, c->d_ynat, c->d_polish};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->search_stream) cudaStreamDestroy(c->search_stream);
    for (auto& e : c->events) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    delete c;
}

int ilog2_exact(int64_t v) {
    if (v <= 0 || (v & (v - 1))) return -1;
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

template <typename T>
int dev_alloc(T** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(FCAS_ERR_NOMEM, "cudaMalloc(%zu bytes) for %s failed: %s", bytes, what, cudaGetErrorString(e));
    }
    return FCAS_OK;
}

// Grow the per-particle buffers to hold n particles.
int ensure_particles(fcas_ctx* c, int64_t n) {
    if (n <= c->params_cap) return FCAS_OK;
    if (c->d_params) cudaFree(c->d_params);
    c->d_params = nullptr;
    c->params_cap = 0;
    int rc = dev_alloc(&c->d_params, sizeof(ParticleParams) * (size_t)n, "particle parameters");
    if (rc) return rc;
    c->params_cap = n;
    return FCAS_OK;
}

int ensure_staging(fcas_ctx* c, int64_t n) {
    if (n <= c->stage_cap) return FCAS_OK;
    if (c->d_theta) cudaFree(c->d_theta);
    if (c->d_fit) cudaFree(c->d_fit);
    if (c->d_tc) cudaFree(c->d_tc);
    c->d_theta = nullptr;
    c->d_fit = nullptr;
    c->d_tc = nullptr;
    c->stage_cap = 0;
    int rc = dev_alloc(&c->d_theta, sizeof(double) * 4 * (size_t)n, "theta staging");
    if (!rc) rc = dev_alloc(&c->d_fit, sizeof(double) * (size_t)n, "fitness staging");
    if (!rc) rc = dev_alloc(&c->d_tc, sizeof(int64_t) * (size_t)n, "tc staging");
    if (rc) return rc;
    c->stage_cap = n;
    return FCAS_OK;
}

void prof_begin(fcas_ctx* c, int kind, cudaStream_t s, size_t* slot) {
    *slot = SIZE_MAX;
    if (!c->prof) return;
    if (c->events_used == c->events.size()) {
        if (c->events.size() >= 65536) return;
        EventPair e;
        if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        c->events.push_back(e);
    }
    *slot = c->events_used++;
    c->events[*slot].kind = kind;
    cudaEventRecord(c->events[*slot].a, s);
}

void prof_end(fcas_ctx* c, size_t slot, cudaStream_t s) {
    if (slot != SIZE_MAX) cudaEventRecord(c->events[slot].b, s);
}

// Passes A, B and the final argmax over chunks of particle parameters, with the given scratch.
cudaError_t launch_passes_with(fcas_ctx* c, const ParticleParams* params, void* inter, Partial* partials,
                               int64_t chunk, int64_t n, double* d_fit, int64_t* d_tc, cudaStream_t st) {
    const FitnessPlan plan = make_plan(c);
    const int prec = c->setup.precision;
    size_t slot;
    cudaError_t e = cudaSuccess;
    for (int64_t p0 = 0; p0 < n && e == cudaSuccess; p0 += chunk) {
        const int64_t np = (n - p0) < chunk ? (n - p0) : chunk;
        prof_begin(c, FCAS_KERNEL_PASS_A, st, &slot);
        e = launch_pass_a_prec(prec, plan, params, p0, np, inter, st);
        prof_end(c, slot, st);
        if (e != cudaSuccess) break;
        prof_begin(c, FCAS_KERNEL_PASS_B, st, &slot);
        e = launch_pass_b_prec(prec, plan, params, p0, np, inter, partials, st);
        prof_end(c, slot, st);
        if (e != cudaSuccess) break;
        prof_begin(c, FCAS_KERNEL_REDUCE, st, &slot);
        e = launch_reduce(partials, c->nb_partials, params, p0, np, d_fit, d_tc, st);
        prof_end(c, slot, st);
    }
    return e;
}

cudaError_t launch_passes(fcas_ctx* c, int64_t n, double* d_fit, int64_t* d_tc, cudaStream_t st) {
    return launch_passes_with(c, c->d_params, c->d_inter, c->d_partials, c->chunk, n, d_fit, d_tc, st);
}

// Per-particle buffers of the adjoint: band sums and a staging array for host outputs.
int ensure_grad(fcas_ctx* c, int64_t n) {
    if (n <= c->grad_cap) return FCAS_OK;
    if (c->d_gsums) cudaFree(c->d_gsums);
    if (c->d_gstage) cudaFree(c->d_gstage);
    c->d_gsums = nullptr;
    c->d_gstage = nullptr;
    c->grad_cap = 0;
    int rc = dev_alloc(&c->d_gsums, sizeof(double) * 12 * (size_t)c->setup.n_det * n, "gradient sums");
    if (!rc) rc = dev_alloc(&c->d_gstage, sizeof(double) * 4 * (size_t)n, "gradient staging");
    if (rc) return rc;
    c->grad_cap = n;
    return FCAS_OK;
}

// d Gamma^2 / d theta at fixed tc for n particles given on the device: geometry into the context's
// particle parameters, the band sums, then their binary64 combination (needs ensure_particles and
// ensure_grad for n).
cudaError_t gradient_device(fcas_ctx* c, int64_t n, const double* d_theta, const int64_t* d_tc, double* d_grad,
                            cudaStream_t st) {
    cudaError_t e = launch_geometry(d_theta, n, c->d_params, c->d_det, c->d_sigma2s, c->setup.n_det, c->setup.f_low,
                                    c->df, pass_a_kstep(c), st);
    if (e != cudaSuccess) return e;
    const FitnessPlan plan = make_plan(c);
    if (c->setup.precision == FCAS_PREC_FP32)
        e = launch_grad_sums<float>(plan, c->k1b, c->k_lo, c->k_hi, c->d_params, d_tc, n, c->d_gsums, st);
    else
        e = launch_grad_sums<double>(plan, c->k1b, c->k_lo, c->k_hi, c->d_params, d_tc, n, c->d_gsums, st,
                                     c->setup.precision == FCAS_PREC_FF);
    if (e != cudaSuccess) return e;
    return launch_grad_final(d_theta, d_tc, n, c->d_gsums, c->d_det, c->d_sigma2s, c->setup.n_det, c->setup.f_low,
                             c->df, d_grad, st);
}

// Scratch of the fitness path (allocated at create unless FCAS_SETUP_LAZY_SCRATCH, else on first use).
int ensure_scratch(fcas_ctx* c) {
    if (c->d_inter) return FCAS_OK;
    const size_t per_particle = inter_bytes_per_particle(c->setup.precision, c->setup.n_fft);
    int rc = dev_alloc(&c->d_inter, per_particle * (size_t)c->chunk, "intermediate transform");
    if (!rc) rc = dev_alloc(&c->d_partials, sizeof(Partial) * (size_t)c->chunk * c->nb_cap, "argmax partials");
    return rc;
}

// Choose the N = N1 N2 split (bias), the pass-A column-block width (k1b; 0 = the default) and the
// CTA grouping (sub), and lay the spectrum out for them.
int apply_layout(fcas_ctx* c, int bias, int k1b, int sub, int radix_bits_a, cudaStream_t st) {
    const int log_n = c->log_n;
    const int l2 = split_log_n2_with(log_n, bias);
    const int l1 = log_n - l2;
    if (l1 > kMaxLogPass) return fail(FCAS_ERR_INVALID, "split bias %d gives a %d-point pass", bias, 1 << l1);
    int ks[8];
    const int nk = pass_a_k1b_variants(l2, c->setup.precision, ks);
    if (nk <= 0) return fail(FCAS_ERR_INVALID, "no pass-A shape for 2^%d-point columns", l2);
    if (k1b == 0) k1b = ks[0];
    bool ok = false;
    if (radix_bits_a == 3) ok = pass_a_radix8_available(l2, c->setup.precision, k1b);
    else for (int q = 0; q < nk; ++q) ok |= ks[q] == k1b;
    if (!ok)
        return fail(FCAS_ERR_INVALID, "pass-A width %d with radix bits %d not compiled for 2^%d-point columns", k1b,
                    radix_bits_a, l2);
    if (sub < 1 || (sub & (sub - 1))) return fail(FCAS_ERR_INVALID, "CTA grouping %d is not a power of two", sub);
    if (radix_bits_a != 4 && !(radix_bits_a == 3 && pass_a_radix8_available(l2, c->setup.precision, k1b)))
        return fail(FCAS_ERR_INVALID, "pass-A radix %d not compiled for this shape", 1 << radix_bits_a);
    const int64_t nb = pass_b_blocks_per_particle(l1, l2, c->setup.precision);
    if (c->nb_cap && nb > c->nb_cap) return fail(FCAS_ERR_INVALID, "split bias %d needs more argmax partials", bias);
    c->split_bias = bias;
    c->log_n2 = l2;
    c->log_n1 = l1;
    c->n1 = (int64_t)1 << l1;
    c->n2 = (int64_t)1 << l2;
    c->k1b = k1b;
    c->sub = sub;
    c->radix_bits_a = radix_bits_a;
    c->nb_partials = nb;
    cudaError_t e = launch_stage_tables(l2, radix_bits_a, c->d_stw_a64, c->d_stw_a32, st);
    if (e == cudaSuccess) e = launch_stage_tables(l1, 4, c->d_stw_b64, c->d_stw_b32, st);
    if (e == cudaSuccess && c->d_stw_aff) e = launch_split_ff(c->d_stw_a64, c->d_stw_aff, (int64_t)1 << l2, st);
    if (e == cudaSuccess && c->d_stw_bff) e = launch_split_ff(c->d_stw_b64, c->d_stw_bff, (int64_t)1 << l1, st);
    if (e == cudaSuccess)
        e = launch_layout(c->d_ynat, c->setup.n_det, log_n, l1, l2, k1b, c->k_lo, c->k_hi, c->setup.fs, c->setup.f_low,
                          c->setup.precision, c->d_y, c->d_basis, st);
    if (e != cudaSuccess) return fail(FCAS_ERR_CUDA, "layout: %s", cudaGetErrorString(e));
    return FCAS_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

int create_impl(fcas_ctx** out, const fcas_setup* setup, const fcas_detector* det, const double* psd,
                const double* data, const int64_t* shifts, void* stream);

}  // namespace

extern "C" {

const char* fcas_last_error(void) { return g_last_error.c_str(); }

int fcas_version(void) { return 100; }

int fcas_create(fcas_ctx** out, const fcas_setup* setup, const fcas_detector* det, const double* psd,
                const double* data, void* stream) {
    NvtxRange nvtx_("fcas_create");
    return create_impl(out, setup, det, psd, data, nullptr, stream);
}

int fcas_create_time_shifted(fcas_ctx** out, const fcas_setup* setup, const fcas_detector* det, const double* psd,
                             const double* data, const int64_t* shifts, void* stream) {
    NvtxRange nvtx_("fcas_create_time_shifted");
    g_last_error.clear();
    if (!shifts) return fail(FCAS_ERR_INVALID, "fcas_create_time_shifted: NULL shifts");
    return create_impl(out, setup, det, psd, data, shifts, stream);
}

}  // extern "C"

namespace {

int create_impl(fcas_ctx** out, const fcas_setup* setup, const fcas_detector* det, const double* psd,
                const double* data, const int64_t* shifts, void* stream) {
    g_last_error.clear();
    if (!out || !setup || !det || !data) return fail(FCAS_ERR_INVALID, "fcas_create: NULL argument");
    *out = nullptr;
    const fcas_setup& s = *setup;
    if (s.n_det < 1 || s.n_det > FCAS_MAX_DET)
        return fail(FCAS_ERR_INVALID, "n_det = %d outside 1..%d", s.n_det, FCAS_MAX_DET);
    if (s.precision != FCAS_PREC_FP32 && s.precision != FCAS_PREC_FP64 && s.precision != FCAS_PREC_FF)
        return fail(FCAS_ERR_INVALID, "precision = %d is not FCAS_PREC_FP32, FCAS_PREC_FP64 or FCAS_PREC_FF",
                    s.precision);
    const int log_n = ilog2_exact(s.n_fft);
    if (log_n < kMinLogN || log_n > kMaxLogN)
        return fail(FCAS_ERR_INVALID, "n_fft = %lld is not a power of two in 2^%d..2^%d", (long long)s.n_fft, kMinLogN,
                    kMaxLogN);
    if (s.n_samples < 1 || s.n_samples > s.n_fft)
        return fail(FCAS_ERR_INVALID, "n_samples = %lld outside 1..n_fft", (long long)s.n_samples);
    if (!(std::isfinite(s.fs) && s.fs > 0.0)) return fail(FCAS_ERR_INVALID, "fs must be finite and > 0");
    if (!(std::isfinite(s.f_low) && std::isfinite(s.f_high) && s.f_low > 0.0 && s.f_high > s.f_low))
        return fail(FCAS_ERR_INVALID, "need 0 < f_low < f_high (finite)");
    if (s.max_batch < 0 || (s.flags & ~FCAS_SETUP_LAZY_SCRATCH) != 0)
        return fail(FCAS_ERR_INVALID, "max_batch < 0 or unknown bits in flags");
    for (int i = 0; i < s.n_det; ++i) {
        const double* v = det[i].r;
        for (int q = 0; q < 9; ++q)
            if (!std::isfinite(v[q])) return fail(FCAS_ERR_INVALID, "detector %d geometry is not finite", i);
        const double nx = std::sqrt(det[i].xarm[0] * det[i].xarm[0] + det[i].xarm[1] * det[i].xarm[1] +
                                    det[i].xarm[2] * det[i].xarm[2]);
        const double ny = std::sqrt(det[i].yarm[0] * det[i].yarm[0] + det[i].yarm[1] * det[i].yarm[1] +
                                    det[i].yarm[2] * det[i].yarm[2]);
        if (std::fabs(nx - 1.0) > 1e-6 || std::fabs(ny - 1.0) > 1e-6)
            return fail(FCAS_ERR_INVALID, "detector %d arm vectors are not unit vectors", i);
    }
    // band: f_low < k fs / N <= f_high, 0 < k < N/2
    const int64_t n = s.n_fft;
    int64_t k_lo = (int64_t)std::floor(s.f_low * (double)n / s.fs) + 1;
    while (k_lo > 1 && (double)(k_lo - 1) * s.fs > s.f_low * (double)n) --k_lo;
    while ((double)k_lo * s.fs <= s.f_low * (double)n) ++k_lo;
    int64_t k_hi = (int64_t)std::floor(s.f_high * (double)n / s.fs);
    while ((double)k_hi * s.fs > s.f_high * (double)n) --k_hi;
    while ((double)(k_hi + 1) * s.fs <= s.f_high * (double)n) ++k_hi;
    if (k_lo < 1) k_lo = 1;
    if (k_hi > n / 2 - 1) k_hi = n / 2 - 1;
    if (k_hi < k_lo) return fail(FCAS_ERR_INVALID, "the band (f_low, f_high] contains no frequency bin");

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return fail(FCAS_ERR_CUDA, "fcas_create: no usable CUDA device");
    }
    fcas_ctx* c = new fcas_ctx();
    c->setup = s;
    c->device = device;
    c->log_n = log_n;
    c->log_n2 = split_log_n2_with(log_n, FCAS_SPLIT_BIAS);
    c->log_n1 = log_n - c->log_n2;
    c->n1 = (int64_t)1 << c->log_n1;
    c->n2 = (int64_t)1 << c->log_n2;
    c->k_lo = k_lo;
    c->k_hi = k_hi;
    c->df = s.fs / (double)n;
    const int D = s.n_det;
    const int64_t psd_row = n / 2 + 1;
    double2* d_spec = nullptr;
    double2* d_work = nullptr;
    double* d_psd = nullptr;
    double* d_data = nullptr;
    double* d_shifted = nullptr;
    int* d_flag = nullptr;
    double* d_sig = nullptr;
    const bool psd_dev = is_device_ptr(psd), data_dev = is_device_ptr(data);
    auto cleanup = [&](int code) {
        if (d_shifted) cudaFree(d_shifted);
        if (d_spec) cudaFree(d_spec);
        if (d_work) cudaFree(d_work);
        if (d_psd && !psd_dev) cudaFree(d_psd);
        if (d_data && !data_dev) cudaFree(d_data);
        if (d_flag) cudaFree(d_flag);
        if (d_sig) cudaFree(d_sig);
        if (code != FCAS_OK) free_ctx(c);
        return code;
    };
#define FCAS_TRY(expr)                      \
    do {                                    \
        int rc_ = (expr);                   \
        if (rc_ != FCAS_OK) return cleanup(rc_); \
    } while (0)
#define FCAS_TRYCUDA(call)                                                                                 \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return cleanup(fail(FCAS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_))); \
    } while (0)

    // inputs on the device (psd = NULL: the analytic aLIGO fit, evaluated on the band bins)
    if (psd_dev) {
        d_psd = const_cast<double*>(psd);
    } else {
        FCAS_TRY(dev_alloc(&d_psd, sizeof(double) * (size_t)D * psd_row, "psd"));
        if (psd)
            FCAS_TRYCUDA(cudaMemcpyAsync(d_psd, psd, sizeof(double) * (size_t)D * psd_row, cudaMemcpyHostToDevice, st));
        else
            FCAS_TRYCUDA(launch_analytic_psd(d_psd, D, psd_row, k_lo, k_hi, c->df, st));
    }
    if (data_dev) {
        d_data = const_cast<double*>(data);
    } else {
        FCAS_TRY(dev_alloc(&d_data, sizeof(double) * (size_t)D * s.n_samples, "data"));
        FCAS_TRYCUDA(cudaMemcpyAsync(d_data, data, sizeof(double) * (size_t)D * s.n_samples, cudaMemcpyHostToDevice,
                                     st));
    }
    if (shifts) {
        // background realisation: each detector's series shifted circularly (the caller's data is
        // left untouched)
        DetShifts sh{};
        for (int i = 0; i < D; ++i) sh.s[i] = ((shifts[i] % s.n_samples) + s.n_samples) % s.n_samples;
        FCAS_TRY(dev_alloc(&d_shifted, sizeof(double) * (size_t)D * s.n_samples, "time-shifted data"));
        FCAS_TRYCUDA(launch_time_shift(d_data, d_shifted, D, s.n_samples, sh, st));
    }
    const double* d_use = shifts ? d_shifted : d_data;
    FCAS_TRY(dev_alloc(&d_flag, sizeof(int), "flag"));
    FCAS_TRYCUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
    FCAS_TRYCUDA(launch_check_finite(d_use, (int64_t)D * s.n_samples, d_flag, st));
    FCAS_TRYCUDA(launch_check_psd(d_psd, D, psd_row, k_lo, k_hi, d_flag, st));
    int h_flag = 0;
    FCAS_TRYCUDA(cudaMemcpyAsync(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    FCAS_TRYCUDA(cudaStreamSynchronize(st));
    if (h_flag & 1) return cleanup(fail(FCAS_ERR_INVALID, "data contains non-finite samples"));
    if (h_flag & 2) return cleanup(fail(FCAS_ERR_INVALID, "psd is non-finite or <= 0 inside the band"));

    // geometry table
    FCAS_TRY(dev_alloc(&c->d_det, sizeof(double) * 9 * D, "detectors"));
    FCAS_TRYCUDA(cudaMemcpyAsync(c->d_det, det, sizeof(double) * 9 * D, cudaMemcpyHostToDevice, st));

    // template norms and the power-of-two scale that brings them near 1
    FCAS_TRY(dev_alloc(&d_sig, sizeof(double) * D * 257, "sigma2"));
    FCAS_TRYCUDA(launch_sigma2(d_psd, D, psd_row, k_lo, k_hi, c->df, d_sig, d_sig + D, st));
    FCAS_TRYCUDA(cudaMemcpyAsync(c->sigma2, d_sig, sizeof(double) * D, cudaMemcpyDeviceToHost, st));
    FCAS_TRYCUDA(cudaStreamSynchronize(st));
    double smax = 0.0;
    for (int i = 0; i < D; ++i) {
        if (!(std::isfinite(c->sigma2[i]) && c->sigma2[i] > 0.0))
            return cleanup(fail(FCAS_ERR_INVALID, "template norm of detector %d is not finite and positive", i));
        smax = std::fmax(smax, c->sigma2[i]);
    }
    c->scale = std::ldexp(1.0, -(int)std::lround(0.5 * std::log2(smax)));
    double s2s[FCAS_MAX_DET];
    for (int i = 0; i < D; ++i) s2s[i] = c->sigma2[i] * c->scale * c->scale;
    FCAS_TRY(dev_alloc(&c->d_sigma2s, sizeof(double) * D, "scaled sigma2"));
    FCAS_TRYCUDA(cudaMemcpyAsync(c->d_sigma2s, s2s, sizeof(double) * D, cudaMemcpyHostToDevice, st));

    // twiddle tables
    const int log_tw = c->log_n1 > c->log_n2 ? c->log_n1 : c->log_n2;
    const size_t ntw = (size_t)1 << log_tw;
    const size_t nlo = (size_t)1 << kTwLoBits;
    const size_t nhi = log_n > kTwLoBits ? ((size_t)1 << (log_n - kTwLoBits)) : 1;
    FCAS_TRY(dev_alloc(&c->d_tw64, sizeof(double2) * ntw, "twiddles"));
    FCAS_TRY(dev_alloc(&c->d_twlo64, sizeof(double2) * nlo, "twiddles"));
    FCAS_TRY(dev_alloc(&c->d_twhi64, sizeof(double2) * nhi, "twiddles"));
    FCAS_TRY(dev_alloc(&c->d_tw32, sizeof(float2) * ntw, "twiddles"));
    FCAS_TRY(dev_alloc(&c->d_twlo32, sizeof(float2) * nlo, "twiddles"));
    FCAS_TRY(dev_alloc(&c->d_twhi32, sizeof(float2) * nhi, "twiddles"));
    FCAS_TRYCUDA(launch_tables(log_n, c->log_n1, c->log_n2, c->d_tw64, c->d_twlo64, c->d_twhi64, c->d_tw32,
                               c->d_twlo32, c->d_twhi32, st));
    const bool fp32 = s.precision == FCAS_PREC_FP32;
    c->d_tw = fp32 ? (void*)c->d_tw32 : (void*)c->d_tw64;
    c->d_twlo = fp32 ? (void*)c->d_twlo32 : (void*)c->d_twlo64;
    c->d_twhi = fp32 ? (void*)c->d_twhi32 : (void*)c->d_twhi64;
    if (s.precision == FCAS_PREC_FF) {
        FCAS_TRY(dev_alloc(&c->d_twloff, sizeof(double2) * nlo, "float-float twiddles"));
        FCAS_TRY(dev_alloc(&c->d_twhiff, sizeof(double2) * nhi, "float-float twiddles"));
        FCAS_TRY(dev_alloc(&c->d_stw_aff, sizeof(double2) << kMaxLogPass, "float-float stage twiddles"));
        FCAS_TRY(dev_alloc(&c->d_stw_bff, sizeof(double2) << kMaxLogPass, "float-float stage twiddles"));
        FCAS_TRYCUDA(launch_split_ff(c->d_twlo64, c->d_twloff, (int64_t)nlo, st));
        FCAS_TRYCUDA(launch_split_ff(c->d_twhi64, c->d_twhiff, (int64_t)nhi, st));
        FCAS_TRY(dev_alloc(&c->d_phff, sizeof(double2) * 1024, "float-float phasor table"));
        FCAS_TRYCUDA(launch_phase_table_ff(c->d_phff, 1024, st));
    }

    // forward FFT of the data (binary64) and the whitened, re-laid-out band spectrum
    FCAS_TRY(dev_alloc(&d_spec, sizeof(double2) * (size_t)D * n, "data spectrum"));
    FCAS_TRY(dev_alloc(&d_work, sizeof(double2) * (size_t)D * n, "data FFT work"));
    FCAS_TRYCUDA(launch_data_fft(d_use, D, s.n_samples, log_n, c->log_n1, c->log_n2, c->d_tw64, log_tw - c->log_n2,
                                 log_tw - c->log_n1, c->d_twlo64, c->d_twhi64, d_work, d_spec, st));
    const size_t half = (size_t)(n / 2);
    FCAS_TRY(dev_alloc(&c->d_ynat, sizeof(double2) * (size_t)D * half, "whitened spectrum (natural order)"));
    FCAS_TRYCUDA(launch_whiten(d_spec, d_psd, D, psd_row, log_n, k_lo, k_hi, s.fs, c->scale, c->d_ynat, st));
    const size_t ysz = (fp32 ? sizeof(float2) : sizeof(double2)) * (size_t)D * half;
    const size_t bsz = (fp32 ? sizeof(BasisF) : sizeof(BasisD)) * half;
    FCAS_TRY(dev_alloc(&c->d_y, ysz, "whitened spectrum"));
    FCAS_TRY(dev_alloc(&c->d_basis, bsz, "chirp basis"));
    FCAS_TRY(dev_alloc(&c->d_stw_a64, sizeof(double2) << kMaxLogPass, "stage twiddles"));
    FCAS_TRY(dev_alloc(&c->d_stw_a32, sizeof(float2) << kMaxLogPass, "stage twiddles"));
    FCAS_TRY(dev_alloc(&c->d_stw_b64, sizeof(double2) << kMaxLogPass, "stage twiddles"));
    FCAS_TRY(dev_alloc(&c->d_stw_b32, sizeof(float2) << kMaxLogPass, "stage twiddles"));
    FCAS_TRY(apply_layout(c, FCAS_SPLIT_BIAS, 0, FCAS_PASS_A_SUB,
                          pass_a_default_radix_bits(split_log_n2_with(c->log_n, FCAS_SPLIT_BIAS), s.precision), st));

    // scratch for the fitness path (partials sized for every split the tuner may choose)
    const size_t per_particle = inter_bytes_per_particle(s.precision, n);
    int64_t chunk = s.max_batch;
    if (chunk == 0) {
        const size_t budget = (size_t)16 << 30;
        chunk = (int64_t)(budget / per_particle);
        if (chunk > 64) chunk = 64;
        if (chunk < 1) chunk = 1;
    }
    c->chunk = chunk;
    c->nb_cap = 0;
    for (int bias = 0; bias <= 1; ++bias) {
        const int l2 = split_log_n2_with(log_n, bias);
        const int64_t nb = pass_b_blocks_per_particle(log_n - l2, l2, s.precision);
        if (nb > c->nb_cap) c->nb_cap = nb;
    }
    if (!(s.flags & FCAS_SETUP_LAZY_SCRATCH)) FCAS_TRY(ensure_scratch(c));
    FCAS_TRYCUDA(cudaStreamSynchronize(st));
#undef FCAS_TRY
#undef FCAS_TRYCUDA
    cleanup(FCAS_OK);
    *out = c;
    return FCAS_OK;
}

}  // namespace

extern "C" {

int fcas_fitness(fcas_ctx* c, int64_t n, const double* theta, double* fitness, int64_t* tc, void* stream) {
    NvtxRange nvtx_("fcas_fitness");
    g_last_error.clear();
    if (!c) return fail(FCAS_ERR_INVALID, "fcas_fitness: NULL context");
    if (n < 0) return fail(FCAS_ERR_INVALID, "fcas_fitness: n < 0");
    if (n == 0) return FCAS_OK;
    if (int rc0 = check_ctx_device(c, "fcas_fitness")) return rc0;
    if (!theta || !fitness || !tc) return fail(FCAS_ERR_INVALID, "fcas_fitness: NULL array");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool th_dev = is_device_ptr(theta), f_dev = is_device_ptr(fitness), t_dev = is_device_ptr(tc);
    if (!th_dev) {
        for (int64_t p = 0; p < n; ++p) {
            const double* t = theta + 4 * p;
            if (!(std::isfinite(t[0]) && std::isfinite(t[1]) && std::isfinite(t[2]) && std::isfinite(t[3]) &&
                  t[2] > 0.0 && t[3] > 0.0))
                return fail(FCAS_ERR_INVALID, "particle %lld: non-finite angle or non-positive chirp time",
                            (long long)p);
        }
    }
    int rc = ensure_particles(c, n);
    if (!rc) rc = ensure_scratch(c);
    if (rc) return rc;
    if (!th_dev || !f_dev || !t_dev) {
        rc = ensure_staging(c, n);
        if (rc) return rc;
    }
    const double* d_theta = theta;
    if (!th_dev) {
        FCAS_CUDA(cudaMemcpyAsync(c->d_theta, theta, sizeof(double) * 4 * (size_t)n, cudaMemcpyHostToDevice, st));
        d_theta = c->d_theta;
    }
    double* d_fit = f_dev ? fitness : c->d_fit;
    int64_t* d_tc = t_dev ? tc : c->d_tc;
    size_t slot;
    prof_begin(c, FCAS_KERNEL_GEOMETRY, st, &slot);
    FCAS_CUDA(launch_geometry(d_theta, n, c->d_params, c->d_det, c->d_sigma2s, c->setup.n_det, c->setup.f_low, c->df,
                              pass_a_kstep(c), st));
    prof_end(c, slot, st);
    FCAS_CUDA(launch_passes(c, n, d_fit, d_tc, st));
    if (!f_dev) FCAS_CUDA(cudaMemcpyAsync(fitness, d_fit, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
    if (!t_dev) FCAS_CUDA(cudaMemcpyAsync(tc, d_tc, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, st));
    if (!th_dev || !f_dev || !t_dev) FCAS_CUDA(cudaStreamSynchronize(st));
    if (const unsigned int bad = take_index_checks(st) | take_index_checks_ff(st))
        return fail(FCAS_ERR_CUDA, "fcas_fitness: index checks failed (bits 0x%x)", bad);
    return FCAS_OK;
}

}  // extern "C"

namespace {

// Device buffers of one swarm: state, parameters, fitness, counters and results.
struct Swarm {
    PsoStateDev s;
    double* theta;
    double* fit;
    int64_t* tcs;
    fcas_search_result* res;
};

size_t swarm_bytes(int64_t rows, int runs) {
    const size_t r4 = align256(sizeof(double) * 4 * rows), r1 = align256(sizeof(double) * rows);
    const size_t ri = align256(sizeof(int64_t) * rows);
    return 4 * r4 + 2 * r1 + 2 * ri + align256(sizeof(int32_t) * runs) + align256(sizeof(int64_t) * runs) +
           align256(sizeof(fcas_search_result) * runs);
}

Swarm carve_swarm(unsigned char* b, int64_t rows, int runs) {
    const size_t r4 = align256(sizeof(double) * 4 * rows), r1 = align256(sizeof(double) * rows);
    const size_t ri = align256(sizeof(int64_t) * rows);
    Swarm w;
    w.s.x = reinterpret_cast<double*>(b);
    w.s.v = reinterpret_cast<double*>(b + r4);
    w.s.pbest_x = reinterpret_cast<double*>(b + 2 * r4);
    w.theta = reinterpret_cast<double*>(b + 3 * r4);
    w.s.pbest_f = reinterpret_cast<double*>(b + 4 * r4);
    w.fit = reinterpret_cast<double*>(b + 4 * r4 + r1);
    w.s.pbest_tc = reinterpret_cast<int64_t*>(b + 4 * r4 + 2 * r1);
    w.tcs = reinterpret_cast<int64_t*>(b + 4 * r4 + 2 * r1 + ri);
    size_t off = 4 * r4 + 2 * r1 + 2 * ri;
    w.s.iter = reinterpret_cast<int32_t*>(b + off);
    off += align256(sizeof(int32_t) * runs);
    w.s.evals = reinterpret_cast<int64_t*>(b + off);
    off += align256(sizeof(int64_t) * runs);
    w.res = reinterpret_cast<fcas_search_result*>(b + off);
    return w;
}

// One PSO iteration of one segment: parameters of the particles inside the box, their fitness, update.
cudaError_t swarm_iteration(fcas_ctx* c, const PsoDev& g, const Swarm& w, ParticleParams* params, void* inter,
                            Partial* partials, int64_t chunk, int64_t rows, cudaStream_t st) {
    cudaError_t x = launch_pso_theta(g, w.s, w.theta, st);
    if (x == cudaSuccess)
        x = launch_geometry(w.theta, rows, params, c->d_det, c->d_sigma2s, c->setup.n_det, c->setup.f_low, c->df,
                            pass_a_kstep(c), st);
    if (x == cudaSuccess) x = launch_passes_with(c, params, inter, partials, chunk, rows, w.fit, w.tcs, st);
    if (x == cudaSuccess) x = launch_pso_update(g, 0, w.fit, w.tcs, w.s, st);
    return x;
}

// Run `iteration` n_iter times on stream st: the first eagerly (it also sets the kernels' shared
// memory attributes), the others as replays of a captured graph of it.
template <typename F>
cudaError_t run_iterations(int n_iter, cudaStream_t st, F&& iteration) {
    cudaError_t e = iteration();
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && n_iter > 1) {
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            cudaError_t ei = iteration();
            e = cudaStreamEndCapture(st, &graph);
            if (e == cudaSuccess) e = ei;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        for (int it = 1; it < n_iter && e == cudaSuccess; ++it) e = cudaGraphLaunch(exec, st);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return e;
}

uint64_t segment_seed(uint64_t seed, int s) { return seed + (uint64_t)s * 0x9E3779B97F4A7C15ull; }

}  // namespace

extern "C" {

int fcas_search(fcas_ctx* c, const fcas_pso_config* cfg, fcas_search_result* results, void* stream) {
    NvtxRange nvtx_("fcas_search");
    g_last_error.clear();
    if (!c || !results) return fail(FCAS_ERR_INVALID, "fcas_search: NULL argument");
    if (int rc0 = check_ctx_device(c, "fcas_search")) return rc0;
    char msg[256];
    int rc = pso_validate(cfg, msg, sizeof(msg));
    if (rc) return fail(rc, "fcas_search: %s", msg);
    const int64_t rows = (int64_t)cfg->n_runs * cfg->n_particles;
    rc = ensure_particles(c, rows);
    if (!rc) rc = ensure_scratch(c);
    if (rc) return rc;
    const size_t need = swarm_bytes(rows, cfg->n_runs);
    if (need > c->pso_bytes) {
        if (c->d_pso) cudaFree(c->d_pso);
        c->d_pso = nullptr;
        c->pso_bytes = 0;
        rc = dev_alloc(&c->d_pso, need, "swarm state");
        if (rc) return rc;
        c->pso_bytes = need;
    }
    const Swarm w = carve_swarm(c->d_pso, rows, cfg->n_runs);
    if (!c->search_stream) FCAS_CUDA(cudaStreamCreateWithFlags(&c->search_stream, cudaStreamNonBlocking));
    cudaStream_t st = c->search_stream;
    cudaEvent_t ev;
    FCAS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, static_cast<cudaStream_t>(stream));
    cudaStreamWaitEvent(st, ev, 0);
    const PsoDev g = pso_dev(cfg);
    const bool prof = c->prof;
    c->prof = false;
    cudaError_t e = launch_pso_init(g, w.s, st);
    if (e == cudaSuccess)
        e = run_iterations(cfg->n_iter, st,
                           [&]() { return swarm_iteration(c, g, w, c->d_params, c->d_inter, c->d_partials, c->chunk,
                                                          rows, st); });
    if (e == cudaSuccess) e = launch_pso_result(g, w.s, w.res, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(results, w.res, sizeof(fcas_search_result) * cfg->n_runs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaEventDestroy(ev);
    c->prof = prof;
    if (e != cudaSuccess) return fail(FCAS_ERR_CUDA, "fcas_search: %s", cudaGetErrorString(e));
    return FCAS_OK;
}

int fcas_autotune(fcas_ctx* c, int64_t n_particles, const char* cache_path, void* stream) {
    NvtxRange nvtx_("fcas_autotune");
    g_last_error.clear();
    if (!c) return fail(FCAS_ERR_INVALID, "fcas_autotune: NULL context");
    if (int rc0 = check_ctx_device(c, "fcas_autotune")) return rc0;
    if (n_particles < 1) return fail(FCAS_ERR_INVALID, "fcas_autotune: n_particles < 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaDeviceProp prop;
    FCAS_CUDA(cudaGetDevice(&dev));
    FCAS_CUDA(cudaGetDeviceProperties(&prop, dev));
    std::string gpu(prop.name);
    for (char& ch : gpu)
        if (ch == ' ') ch = '_';
    char key[512];
    snprintf(key, sizeof(key), "fcas-tune-v3 %s %lld %d %d %lld", gpu.c_str(), (long long)c->setup.n_fft,
             c->setup.n_det, c->setup.precision, (long long)n_particles);
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[1024];
            while (fgets(line, sizeof(line), f)) {
                if (strncmp(line, key, strlen(key)) != 0 || line[strlen(key)] != ' ') continue;
                int bias, k1b, sub, rbits;
                double ms;
                if (sscanf(line + strlen(key), "%d %d %d %d %lf", &bias, &k1b, &sub, &rbits, &ms) == 5) {
                    fclose(f);
                    int rc = apply_layout(c, bias, k1b, sub, rbits, st);
                    if (rc) return rc;
                    c->tuned_ms = ms;
                    FCAS_CUDA(cudaStreamSynchronize(st));
                    return FCAS_OK;
                }
            }
            fclose(f);
        }
    }
    int rc = ensure_particles(c, n_particles);
    if (!rc) rc = ensure_scratch(c);
    if (!rc) rc = ensure_staging(c, n_particles);
    if (rc) return rc;
    std::vector<double> th(4 * (size_t)n_particles);
    for (int64_t p = 0; p < n_particles; ++p) {   // any valid parameters: the cost does not depend on them
        th[4 * p + 0] = 0.1 * (double)(p % 60);
        th[4 * p + 1] = -1.2 + 0.04 * (double)(p % 60);
        th[4 * p + 2] = 1.0 + 0.01 * (double)(p % 50);
        th[4 * p + 3] = 0.1 + 0.001 * (double)(p % 50);
    }
    FCAS_CUDA(cudaMemcpyAsync(c->d_theta, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, st));
    FCAS_CUDA(launch_geometry(c->d_theta, n_particles, c->d_params, c->d_det, c->d_sigma2s, c->setup.n_det,
                              c->setup.f_low, c->df, pass_a_kstep(c), st));
    cudaEvent_t e0, e1;
    FCAS_CUDA(cudaEventCreate(&e0));
    FCAS_CUDA(cudaEventCreate(&e1));
    const bool prof = c->prof;
    c->prof = false;
    double best_ms = 1e300;
    int best_bias = c->split_bias, best_k = c->k1b, best_sub = c->sub, best_rb = c->radix_bits_a;
    int last_l2 = -1;
    const int subs[4] = {1, 4, 8, 16};
    for (int bias = 0; bias <= 1 && rc == FCAS_OK; ++bias) {
        const int l2 = split_log_n2_with(c->log_n, bias);
        if (l2 == last_l2 || c->log_n - l2 > kMaxLogPass) continue;
        last_l2 = l2;
        int ks[8], rbs[8];
        int nk = pass_a_k1b_variants(l2, c->setup.precision, ks);   // at most 4, plus 2 radix-8 shapes below
        for (int q = 0; q < nk; ++q) rbs[q] = 4;
        for (int k8 : {4, 2}) {
            if (pass_a_radix8_available(l2, c->setup.precision, k8)) {
                ks[nk] = k8;
                rbs[nk++] = 3;
            }
        }
        for (int q = 0; q < nk && rc == FCAS_OK; ++q) {
            for (int si = 0; si < 4 && rc == FCAS_OK; ++si) {
                rc = apply_layout(c, bias, ks[q], subs[si], rbs[q], st);
                if (rc) break;
                cudaError_t e = launch_passes(c, n_particles, c->d_fit, c->d_tc, st);   // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_passes(c, n_particles, c->d_fit, c->d_tc, st);
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    rc = fail(FCAS_ERR_CUDA, "fcas_autotune: %s", cudaGetErrorString(e));
                    break;
                }
                const double per = ms / 3.0 / (double)n_particles;
                if (per < best_ms) {
                    best_ms = per;
                    best_bias = bias;
                    best_k = ks[q];
                    best_sub = subs[si];
                    best_rb = rbs[q];
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->prof = prof;
    if (rc) return rc;
    rc = apply_layout(c, best_bias, best_k, best_sub, best_rb, st);
    if (rc) return rc;
    c->tuned_ms = best_ms;
    FCAS_CUDA(cudaStreamSynchronize(st));
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s %d %d %d %d %.9g\n", key, best_bias, best_k, best_sub, best_rb, best_ms);
            fclose(f);
        }
    }
    return FCAS_OK;
}

int fcas_set_shape(fcas_ctx* c, int32_t split_bias, int32_t k1b, int32_t sub, int32_t radix_bits_a, void* stream) {
    g_last_error.clear();
    if (!c) return fail(FCAS_ERR_INVALID, "fcas_set_shape: NULL context");
    if (int rc0 = check_ctx_device(c, "fcas_set_shape")) return rc0;
    if (split_bias < 0 || split_bias > 1) return fail(FCAS_ERR_INVALID, "fcas_set_shape: split_bias must be 0 or 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (radix_bits_a == 0) radix_bits_a = pass_a_default_radix_bits(split_log_n2_with(c->log_n, split_bias),
                                                                     c->setup.precision);
    int rc = apply_layout(c, split_bias, k1b, sub, radix_bits_a, st);
    if (rc) return rc;
    c->tuned_ms = 0.0;
    FCAS_CUDA(cudaStreamSynchronize(st));
    return FCAS_OK;
}

}  // extern "C"

struct fcas_group {
    std::vector<fcas_ctx*> ctxs;
    int64_t chunk = 0;
    void* d_inter = nullptr;
    Partial* d_partials = nullptr;
    ParticleParams* d_params = nullptr;
    int64_t params_cap = 0;
    unsigned char* d_pso = nullptr;
    size_t pso_bytes = 0;
    cudaStream_t st = nullptr;
};

extern "C" {

int fcas_group_create(fcas_group** out, int32_t n_ctx, fcas_ctx* const* ctxs, int32_t max_batch) {
    g_last_error.clear();
    if (!out || !ctxs || n_ctx < 1) return fail(FCAS_ERR_INVALID, "fcas_group_create: need n_ctx >= 1 contexts");
    if (max_batch < 0) return fail(FCAS_ERR_INVALID, "fcas_group_create: max_batch < 0");
    *out = nullptr;
    size_t inter_pp = 0;
    int64_t nb = 0;
    for (int i = 0; i < n_ctx; ++i) {
        if (!ctxs[i]) return fail(FCAS_ERR_INVALID, "fcas_group_create: context %d is NULL", i);
        if (int rc0 = check_ctx_device(ctxs[i], "fcas_group_create")) return rc0;
        const size_t b = inter_bytes_per_particle(ctxs[i]->setup.precision, ctxs[i]->setup.n_fft);
        if (b > inter_pp) inter_pp = b;
        if (ctxs[i]->nb_cap > nb) nb = ctxs[i]->nb_cap;
    }
    fcas_group* g = new fcas_group();
    g->ctxs.assign(ctxs, ctxs + n_ctx);
    int64_t chunk = max_batch;
    if (chunk == 0) chunk = std::max<int64_t>(1, std::min<int64_t>(64, (int64_t)(((size_t)16 << 30) / inter_pp)));
    g->chunk = chunk;
    int rc = dev_alloc(&g->d_inter, inter_pp * (size_t)chunk, "group intermediate transform");
    if (!rc) rc = dev_alloc(&g->d_partials, sizeof(Partial) * (size_t)chunk * nb, "group argmax partials");
    if (!rc) {
        cudaError_t e = cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = fail(FCAS_ERR_CUDA, "fcas_group_create: %s", cudaGetErrorString(e));
    }
    if (rc) {
        fcas_group_destroy(g);
        return rc;
    }
    *out = g;
    return FCAS_OK;
}

int fcas_group_search(fcas_group* g, const fcas_pso_config* cfg, fcas_search_result* results, void* stream) {
    return fcas_group_search_boxes(g, cfg, nullptr, results, stream);
}

int fcas_group_search_boxes(fcas_group* g, const fcas_pso_config* cfg, const double* boxes,
                            fcas_search_result* results, void* stream) {
    NvtxRange nvtx_("fcas_group_search");
    g_last_error.clear();
    if (!g || !results) return fail(FCAS_ERR_INVALID, "fcas_group_search: NULL argument");
    for (const fcas_ctx* c : g->ctxs)
        if (int rc0 = check_ctx_device(c, "fcas_group_search")) return rc0;
    char msg[256];
    int rc = pso_validate(cfg, msg, sizeof(msg));
    if (rc) return fail(rc, "fcas_group_search: %s", msg);
    const int n_ctx = (int)g->ctxs.size();
    std::vector<fcas_pso_config> cfgs(n_ctx, *cfg);
    for (int i = 0; i < n_ctx; ++i) {
        cfgs[i].seed = segment_seed(cfg->seed, i);
        if (boxes) {
            for (int d = 0; d < 8; ++d) cfgs[i].box[d] = boxes[8 * i + d];
            rc = pso_validate(&cfgs[i], msg, sizeof(msg));
            if (rc) return fail(rc, "fcas_group_search_boxes: segment %d: %s", i, msg);
        }
    }
    const int64_t rows = (int64_t)cfg->n_runs * cfg->n_particles;
    if (rows > g->params_cap) {
        if (g->d_params) cudaFree(g->d_params);
        g->d_params = nullptr;
        g->params_cap = 0;
        rc = dev_alloc(&g->d_params, sizeof(ParticleParams) * (size_t)rows, "group particle parameters");
        if (rc) return rc;
        g->params_cap = rows;
    }
    const size_t per = align256(swarm_bytes(rows, cfg->n_runs));
    if (per * n_ctx > g->pso_bytes) {
        if (g->d_pso) cudaFree(g->d_pso);
        g->d_pso = nullptr;
        g->pso_bytes = 0;
        rc = dev_alloc(&g->d_pso, per * n_ctx, "group swarm state");
        if (rc) return rc;
        g->pso_bytes = per * n_ctx;
    }
    std::vector<Swarm> ws(n_ctx);
    std::vector<PsoDev> gs(n_ctx);
    for (int i = 0; i < n_ctx; ++i) {
        ws[i] = carve_swarm(g->d_pso + per * i, rows, cfg->n_runs);
        gs[i] = pso_dev(&cfgs[i]);
    }
    cudaStream_t st = g->st;
    cudaEvent_t ev;
    FCAS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, static_cast<cudaStream_t>(stream));
    cudaStreamWaitEvent(st, ev, 0);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n_ctx && e == cudaSuccess; ++i) e = launch_pso_init(gs[i], ws[i].s, st);
    if (e == cudaSuccess)
        e = run_iterations(cfg->n_iter, st, [&]() {
            cudaError_t x = cudaSuccess;
            for (int i = 0; i < n_ctx && x == cudaSuccess; ++i)
                x = swarm_iteration(g->ctxs[i], gs[i], ws[i], g->d_params, g->d_inter, g->d_partials, g->chunk, rows,
                                    st);
            return x;
        });
    for (int i = 0; i < n_ctx && e == cudaSuccess; ++i) {
        e = launch_pso_result(gs[i], ws[i].s, ws[i].res, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(results + (size_t)i * cfg->n_runs, ws[i].res, sizeof(fcas_search_result) * cfg->n_runs,
                                cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return fail(FCAS_ERR_CUDA, "fcas_group_search: %s", cudaGetErrorString(e));
    return FCAS_OK;
}

int fcas_tau_tiles(double tau0_lo, double tau0_hi, double tau15_lo, double tau15_hi, int32_t n0, int32_t n15,
                   double overlap, double* boxes) {
    g_last_error.clear();
    if (!boxes) return fail(FCAS_ERR_INVALID, "fcas_tau_tiles: NULL boxes");
    if (n0 < 1 || n15 < 1) return fail(FCAS_ERR_INVALID, "fcas_tau_tiles: need n0, n15 >= 1");
    if (!(overlap >= 0.0 && overlap < 1.0)) return fail(FCAS_ERR_INVALID, "fcas_tau_tiles: need 0 <= overlap < 1");
    if (!(std::isfinite(tau0_lo) && std::isfinite(tau0_hi) && std::isfinite(tau15_lo) && std::isfinite(tau15_hi) &&
          tau0_lo > 0.0 && tau15_lo > 0.0 && tau0_hi > tau0_lo && tau15_hi > tau15_lo))
        return fail(FCAS_ERR_INVALID, "fcas_tau_tiles: need finite 0 < lo < hi on both axes");
    const double w0 = (tau0_hi - tau0_lo) / ((double)n0 - (double)(n0 - 1) * overlap);
    const double w15 = (tau15_hi - tau15_lo) / ((double)n15 - (double)(n15 - 1) * overlap);
    const double kPi = 3.14159265358979323846;
    for (int a = 0; a < n0; ++a) {
        for (int b = 0; b < n15; ++b) {
            double* bx = boxes + 8 * ((int64_t)a * n15 + b);
            bx[0] = 0.0;
            bx[1] = 2.0 * kPi;
            bx[2] = -0.5 * kPi;
            bx[3] = 0.5 * kPi;
            bx[4] = tau0_lo + a * (1.0 - overlap) * w0;
            bx[5] = a == n0 - 1 ? tau0_hi : bx[4] + w0;
            bx[6] = tau15_lo + b * (1.0 - overlap) * w15;
            bx[7] = b == n15 - 1 ? tau15_hi : bx[6] + w15;
        }
    }
    return FCAS_OK;
}

void fcas_group_destroy(fcas_group* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    void* ptrs[] = {g->d_inter, g->d_partials, g->d_params, g->d_pso};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (g->st) cudaStreamDestroy(g->st);
    delete g;
}

int fcas_gradient(fcas_ctx* c, int64_t n, const double* theta, const int64_t* tc, double* grad, void* stream) {
    NvtxRange nvtx_("fcas_gradient");
    g_last_error.clear();
    if (!c) return fail(FCAS_ERR_INVALID, "fcas_gradient: NULL context");
    if (n < 0) return fail(FCAS_ERR_INVALID, "fcas_gradient: n < 0");
    if (n == 0) return FCAS_OK;
    if (int rc0 = check_ctx_device(c, "fcas_gradient")) return rc0;
    if (!theta || !tc || !grad) return fail(FCAS_ERR_INVALID, "fcas_gradient: NULL array");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool th_dev = is_device_ptr(theta), tc_dev = is_device_ptr(tc), g_dev = is_device_ptr(grad);
    int rc = ensure_particles(c, n);
    if (!rc) rc = ensure_grad(c, n);
    if (rc) return rc;
    if (!th_dev || !tc_dev) {
        rc = ensure_staging(c, n);
        if (rc) return rc;
    }
    const double* d_theta = theta;
    if (!th_dev) {
        FCAS_CUDA(cudaMemcpyAsync(c->d_theta, theta, sizeof(double) * 4 * (size_t)n, cudaMemcpyHostToDevice, st));
        d_theta = c->d_theta;
    }
    const int64_t* d_tc = tc;
    if (!tc_dev) {
        FCAS_CUDA(cudaMemcpyAsync(c->d_tc, tc, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, st));
        d_tc = c->d_tc;
    }
    double* d_grad = g_dev ? grad : c->d_gstage;
    FCAS_CUDA(gradient_device(c, n, d_theta, d_tc, d_grad, st));
    if (!g_dev) {
        FCAS_CUDA(cudaMemcpyAsync(grad, d_grad, sizeof(double) * 4 * (size_t)n, cudaMemcpyDeviceToHost, st));
    }
    if (!th_dev || !tc_dev || !g_dev) FCAS_CUDA(cudaStreamSynchronize(st));
    return FCAS_OK;
}

int fcas_polish(fcas_ctx* c, int64_t n, double* theta, double* fitness, int64_t* tc, int32_t steps,
                const double* scales, int32_t max_halvings, int32_t* accepted, void* stream) {
    NvtxRange nvtx_("fcas_polish");
    g_last_error.clear();
    if (!c) return fail(FCAS_ERR_INVALID, "fcas_polish: NULL context");
    if (n < 0 || steps < 0 || max_halvings < 1)
        return fail(FCAS_ERR_INVALID, "fcas_polish: need n >= 0, steps >= 0 and max_halvings >= 1");
    if (n == 0) return FCAS_OK;
    if (int rc0 = check_ctx_device(c, "fcas_polish")) return rc0;
    if (!theta || !fitness || !tc) return fail(FCAS_ERR_INVALID, "fcas_polish: NULL array");
    PolishScales sc{{1e-2, 1e-2, 1e-4, 1e-4}};
    if (scales) {
        for (int m = 0; m < 4; ++m) {
            if (!(std::isfinite(scales[m]) && scales[m] > 0.0))
                return fail(FCAS_ERR_INVALID, "fcas_polish: scales must be finite and > 0");
            sc.s[m] = scales[m];
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool th_dev = is_device_ptr(theta), f_dev = is_device_ptr(fitness), t_dev = is_device_ptr(tc);
    const bool a_dev = accepted && is_device_ptr(accepted);
    int rc = ensure_particles(c, n);
    if (!rc) rc = ensure_scratch(c);
    if (!rc) rc = ensure_grad(c, n);
    if (rc) return rc;
    // working arrays: theta, trial points, directions, gradients [n][4]; fitness, trial fitness and step
    // lengths [n]; tc and trial tc [n]; done and accepted flags [n]; the count of particles still searching
    const size_t r4 = align256(sizeof(double) * 4 * n), r1 = align256(sizeof(double) * n);
    const size_t ri = align256(sizeof(int64_t) * n), rf = align256(sizeof(int32_t) * n);
    const size_t need = 4 * r4 + 3 * r1 + 2 * ri + 2 * rf + 256;
    if (need > c->polish_bytes) {
        if (c->d_polish) cudaFree(c->d_polish);
        c->d_polish = nullptr;
        c->polish_bytes = 0;
        rc = dev_alloc(&c->d_polish, need, "polishing buffers");
        if (rc) return rc;
        c->polish_bytes = need;
    }
    unsigned char* b = c->d_polish;
    double* w_th = reinterpret_cast<double*>(b);
    double* w_cand = reinterpret_cast<double*>(b + r4);
    double* w_dir = reinterpret_cast<double*>(b + 2 * r4);
    double* w_grad = reinterpret_cast<double*>(b + 3 * r4);
    double* w_fit = reinterpret_cast<double*>(b + 4 * r4);
    double* w_cfit = reinterpret_cast<double*>(b + 4 * r4 + r1);
    double* w_step = reinterpret_cast<double*>(b + 4 * r4 + 2 * r1);
    int64_t* w_tc = reinterpret_cast<int64_t*>(b + 4 * r4 + 3 * r1);
    int64_t* w_ctc = reinterpret_cast<int64_t*>(b + 4 * r4 + 3 * r1 + ri);
    int32_t* w_done = reinterpret_cast<int32_t*>(b + 4 * r4 + 3 * r1 + 2 * ri);
    int32_t* w_acc = reinterpret_cast<int32_t*>(b + 4 * r4 + 3 * r1 + 2 * ri + rf);
    int32_t* w_searching = reinterpret_cast<int32_t*>(b + 4 * r4 + 3 * r1 + 2 * ri + 2 * rf);

    FCAS_CUDA(cudaMemcpyAsync(w_th, theta, sizeof(double) * 4 * (size_t)n,
                              th_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    FCAS_CUDA(cudaMemsetAsync(w_acc, 0, sizeof(int32_t) * (size_t)n, st));
    // the fitness at the starting points
    FCAS_CUDA(launch_geometry(w_th, n, c->d_params, c->d_det, c->d_sigma2s, c->setup.n_det, c->setup.f_low, c->df,
                              pass_a_kstep(c), st));
    FCAS_CUDA(launch_passes(c, n, w_fit, w_tc, st));
    for (int32_t step = 0; step < steps; ++step) {
        FCAS_CUDA(gradient_device(c, n, w_th, w_tc, w_grad, st));
        FCAS_CUDA(launch_polish_direction(w_th, w_grad, sc, n, w_dir, w_step, w_done, st));
        for (int32_t h = 0; h < max_halvings; ++h) {
            FCAS_CUDA(cudaMemsetAsync(w_searching, 0, sizeof(int32_t), st));
            FCAS_CUDA(launch_polish_candidate(w_th, w_dir, w_step, w_done, n, w_cand, st));
            FCAS_CUDA(launch_geometry(w_cand, n, c->d_params, c->d_det, c->d_sigma2s, c->setup.n_det, c->setup.f_low,
                                      c->df, pass_a_kstep(c), st));
            FCAS_CUDA(launch_passes(c, n, w_cfit, w_ctc, st));
            FCAS_CUDA(launch_polish_accept(w_th, w_fit, w_tc, w_cand, w_cfit, w_ctc, w_step, w_done, w_acc, n,
                                           w_searching, st));
            int32_t searching = 0;
            FCAS_CUDA(cudaMemcpyAsync(&searching, w_searching, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            FCAS_CUDA(cudaStreamSynchronize(st));
            if (searching == 0) break;
        }
    }
    FCAS_CUDA(cudaMemcpyAsync(theta, w_th, sizeof(double) * 4 * (size_t)n,
                              th_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    FCAS_CUDA(cudaMemcpyAsync(fitness, w_fit, sizeof(double) * (size_t)n,
                              f_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    FCAS_CUDA(cudaMemcpyAsync(tc, w_tc, sizeof(int64_t) * (size_t)n,
                              t_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (accepted)
        FCAS_CUDA(cudaMemcpyAsync(accepted, w_acc, sizeof(int32_t) * (size_t)n,
                                  a_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    FCAS_CUDA(cudaStreamSynchronize(st));
    if (const unsigned int bad = take_index_checks(st) | take_index_checks_ff(st))
        return fail(FCAS_ERR_CUDA, "fcas_polish: index checks failed (bits 0x%x)", bad);
    return FCAS_OK;
}

int fcas_condition_number(fcas_ctx* c, int64_t n, const double* theta, double* kappa, void* stream) {
    g_last_error.clear();
    if (!c) return fail(FCAS_ERR_INVALID, "fcas_condition_number: NULL context");
    if (n < 0) return fail(FCAS_ERR_INVALID, "fcas_condition_number: n < 0");
    if (n == 0) return FCAS_OK;
    if (int rc0 = check_ctx_device(c, "fcas_condition_number")) return rc0;
    if (!theta || !kappa) return fail(FCAS_ERR_INVALID, "fcas_condition_number: NULL array");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool th_dev = is_device_ptr(theta), k_dev = is_device_ptr(kappa);
    if (!th_dev || !k_dev) {
        const int rc = ensure_staging(c, n);
        if (rc) return rc;
    }
    const double* d_theta = theta;
    if (!th_dev) {
        FCAS_CUDA(cudaMemcpyAsync(c->d_theta, theta, sizeof(double) * 4 * (size_t)n, cudaMemcpyHostToDevice, st));
        d_theta = c->d_theta;
    }
    double* d_kappa = k_dev ? kappa : c->d_fit;
    FCAS_CUDA(launch_condition(d_theta, n, c->d_det, c->setup.n_det, d_kappa, st));
    if (!k_dev) {
        FCAS_CUDA(cudaMemcpyAsync(kappa, d_kappa, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
        FCAS_CUDA(cudaStreamSynchronize(st));
    }
    return FCAS_OK;
}

void fcas_destroy(fcas_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    free_ctx(c);
}

int fcas_get_info(const fcas_ctx* c, fcas_info* info) {
    if (!c || !info) return fail(FCAS_ERR_INVALID, "fcas_get_info: NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->n_fft = c->setup.n_fft;
    info->n1 = c->n1;
    info->n2 = c->n2;
    info->k_lo = c->k_lo;
    info->k_hi = c->k_hi;
    info->n_band = c->k_hi - c->k_lo + 1;
    info->chunk = c->chunk;
    info->n_det = c->setup.n_det;
    info->precision = c->setup.precision;
    info->scale = c->scale;
    for (int i = 0; i < c->setup.n_det; ++i) info->sigma2[i] = c->sigma2[i];
    info->inter_bytes = (int64_t)inter_bytes_per_particle(c->setup.precision, c->setup.n_fft);
    info->series = kSeries;
    info->split_bias = c->split_bias;
    info->k1b = c->k1b;
    info->sub = c->sub;
    info->radix_bits_a = c->radix_bits_a;
    info->tuned_ms_per_particle = c->tuned_ms;
    return FCAS_OK;
}

int fcas_profile_enable(fcas_ctx* c, int on) {
    if (!c) return fail(FCAS_ERR_INVALID, "fcas_profile_enable: NULL context");
    c->prof = on != 0;
    c->events_used = 0;
    return FCAS_OK;
}

int fcas_profile_read(fcas_ctx* c, int kind, double* total_ms, int64_t* launches) {
    if (!c || !total_ms || !launches) return fail(FCAS_ERR_INVALID, "fcas_profile_read: NULL argument");
    if (kind < 0 || kind >= FCAS_KERNEL_KINDS) return fail(FCAS_ERR_INVALID, "unknown kernel kind %d", kind);
    double sum = 0.0;
    int64_t cnt = 0;
    for (size_t i = 0; i < c->events_used; ++i) {
        if (c->events[i].kind != kind) continue;
        FCAS_CUDA(cudaEventSynchronize(c->events[i].b));
        float ms = 0.f;
        FCAS_CUDA(cudaEventElapsedTime(&ms, c->events[i].a, c->events[i].b));
        sum += ms;
        ++cnt;
    }
    *total_ms = sum;
    *launches = cnt;
    return FCAS_OK;
}

}  // extern "C"
