// fcas_fitness_noalloc: the fitness evaluation of fcas_fitness with its per-call scratch (particle
// parameters, the intermediate transform between the two FFT passes and the argmax partials)
// placed in one file-scope device array instead of memory allocated by the context. It serves
// callers that must not allocate device memory once their analysis loop runs (see include/fcas.h).
#include <cmath>
#include <cstdio>
#include <mutex>

#include "fcas_ctx.cuh"

namespace {
// 32 MiB, allocated on a device when this module is loaded there (lazily: at the first call of the
// entry point on that device) and held until the process exits
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;
}  // namespace

// The scratch itself. In host code this name is only a stand-in for the device array: kernels must
// receive the address returned by cudaGetSymbolAddress for the current device.
static __device__ __align__(256) unsigned char g_fcas_static_scratch[kStaticScratchBytes];

namespace {

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: look up the device address of the scratch array.
int scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fcas::report_error(FCAS_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fcas::report_error(FCAS_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fcas_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            char msg[256];
            snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return fcas::report_error(FCAS_ERR_CUDA, msg);
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FCAS_OK;
}

size_t round256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

extern "C" int fcas_fitness_noalloc(const fcas_ctx* c, int64_t n, const double* theta, double* fitness, int64_t* tc,
                                    void* stream) {
    using namespace fcas;
    if (!c) return report_error(FCAS_ERR_INVALID, "fcas_fitness_noalloc: NULL context");
    if (n < 0) return report_error(FCAS_ERR_INVALID, "fcas_fitness_noalloc: n < 0");
    if (n == 0) return FCAS_OK;
    if (!theta || !fitness || !tc) return report_error(FCAS_ERR_INVALID, "fcas_fitness_noalloc: NULL array");
    // the context, the arrays, the scratch address and the stream must all belong to the current device
    int rc = check_ctx_device(c, "fcas_fitness_noalloc");
    if (rc == FCAS_OK) rc = check_device_array(theta, "fcas_fitness_noalloc", "theta");
    if (rc == FCAS_OK) rc = check_device_array(fitness, "fcas_fitness_noalloc", "fitness");
    if (rc == FCAS_OK) rc = check_device_array(tc, "fcas_fitness_noalloc", "tc");
    if (rc != FCAS_OK) return rc;
    void* base = nullptr;
    rc = scratch_address(&base);
    if (rc != FCAS_OK) return rc;

    const bool fp32 = c->setup.precision == FCAS_PREC_FP32;
    const size_t inter_pp = inter_bytes_per_particle(c->setup.precision, c->setup.n_fft);
    const size_t part_pp = sizeof(Partial) * (size_t)c->nb_partials;
    const size_t per_particle = sizeof(ParticleParams) + part_pp + inter_pp;
    const size_t usable = kStaticScratchBytes - 3 * 256;
    const int64_t cap = (int64_t)(usable / per_particle);
    if (cap < 1) {
        char msg[320];
        snprintf(msg, sizeof(msg),
                 "fcas_fitness_noalloc: one particle needs %zu bytes of scratch (n_det = %d, n_fft = %lld, %s) but the "
                 "static scratch holds %zu bytes; use fcas_fitness for this segment",
                 per_particle, c->setup.n_det, (long long)c->setup.n_fft, fp32 ? "FP32" : "FP64/FF", kStaticScratchBytes);
        return report_error(FCAS_ERR_INVALID, msg);
    }
    // scratch layout for `cap` particles: parameters | argmax partials | intermediate transform.
    // Nothing in it needs to start at zero: every word a kernel reads is written earlier in the same call.
    unsigned char* b = static_cast<unsigned char*>(base);
    ParticleParams* params = reinterpret_cast<ParticleParams*>(b);
    Partial* partials = reinterpret_cast<Partial*>(b + round256(sizeof(ParticleParams) * cap));
    void* inter = b + round256(sizeof(ParticleParams) * cap) + round256(part_pp * cap);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const FitnessPlan plan = make_plan(c);
    cudaError_t e = cudaSuccess;
    for (int64_t p0 = 0; p0 < n && e == cudaSuccess; p0 += cap) {
        const int64_t np = (n - p0) < cap ? (n - p0) : cap;
        e = launch_geometry(theta + 4 * p0, np, params, c->d_det, c->d_sigma2s, c->setup.n_det, c->setup.f_low, c->df,
                            pass_a_kstep(c), st);
        if (e == cudaSuccess)
            e = launch_pass_a_prec(c->setup.precision, plan, params, 0, np, inter, st);
        if (e == cudaSuccess) e = launch_pass_b_prec(c->setup.precision, plan, params, 0, np, inter, partials, st);
        if (e == cudaSuccess) e = launch_reduce(partials, c->nb_partials, params, 0, np, fitness + p0, tc + p0, st);
    }
    if (e != cudaSuccess) return report_error(FCAS_ERR_CUDA, cudaGetErrorString(e));
    // checked build (FCAS_CHECKED): wait for the launches and report a failed index check as this
    // call's failure; other builds return at once
    if (const unsigned int bad = take_index_checks(st) | take_index_checks_ff(st)) {
        char msg[96];
        snprintf(msg, sizeof(msg), "fcas_fitness_noalloc: index checks failed (bits 0x%x)", bad);
        return report_error(FCAS_ERR_CUDA, msg);
    }
    return FCAS_OK;
}
