// Device-resident lbest particle swarm (Sec. III): Philox4x32-10 random numbers, initialisation,
// positions -> parameters, personal/local-best update and move, per-run results. The move is
// evaluated in binary64 with explicitly rounded operations (no contraction into fused
// multiply-adds) in the order documented in include/fcas.h, so it is reproducible bit for bit.
#include <cfloat>
#include <cmath>
#include <cstdio>

#include "fcas_ctx.cuh"
#include "fcas_pso.cuh"

namespace fcas {

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round multiplies counter
// words 0 and 2 by fixed 32-bit constants, mixes the high halves with words 1, 3 and the key,
// and the key advances by a Weyl sequence between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        if (r < 9) {
            k.x += W0;
            k.y += W1;
        }
    }
    return c;
}

__device__ __forceinline__ double u01(uint32_t u) {
    return __dmul_rn(__dadd_rn((double)u, 0.5), 2.3283064365386963e-10);   // (u + 1/2) 2^-32, exact
}

__device__ __forceinline__ void draw4(const PsoDev& g, uint32_t run, uint32_t it, uint32_t p, uint32_t stream,
                                      double out[4]) {
    const uint4 r = philox4x32_10(make_uint4(run, it, p, stream), make_uint2(g.key0, g.key1));
    out[0] = u01(r.x);
    out[1] = u01(r.y);
    out[2] = u01(r.z);
    out[3] = u01(r.w);
}

__device__ __forceinline__ bool in_box(const double* x) {
    return x[0] >= 0.0 && x[0] <= 1.0 && x[1] >= 0.0 && x[1] <= 1.0 && x[2] >= 0.0 && x[2] <= 1.0 && x[3] >= 0.0 &&
           x[3] <= 1.0;
}

__global__ void pso_init_kernel(PsoDev g, PsoStateDev s) {
    const int64_t rows = (int64_t)g.n_runs * g.n_particles;
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    const uint32_t run = (uint32_t)(row / g.n_particles), p = (uint32_t)(row % g.n_particles);
    double x[4], u[4];
    draw4(g, run, 0xFFFFFFFFu, p, 0, x);
    draw4(g, run, 0xFFFFFFFFu, p, 1, u);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        s.x[4 * row + d] = x[d];
        s.pbest_x[4 * row + d] = x[d];
        s.v[4 * row + d] = fmin(fmax(__dsub_rn(u[d], x[d]), -g.vmax), g.vmax);
    }
    s.pbest_f[row] = -INFINITY;
    s.pbest_tc[row] = -1;
    if (p == 0) {
        if (s.iter) s.iter[run] = 0;
        if (s.evals) s.evals[run] = 0;
    }
}

// Parameters of every particle; NaN outside the box so that the fitness path skips it.
__global__ void pso_theta_kernel(PsoDev g, PsoStateDev s, double* __restrict__ theta) {
    const int64_t rows = (int64_t)g.n_runs * g.n_particles;
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    double x[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) x[d] = s.x[4 * row + d];
    const bool inside = in_box(x);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const double lo = g.box[2 * d], hi = g.box[2 * d + 1];
        theta[4 * row + d] = inside ? __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), x[d])) : NAN;
    }
}

// One CTA per run, one thread per particle.
__global__ void pso_update_kernel(PsoDev g, int32_t iter_arg, const double* __restrict__ fitness,
                                  const int64_t* __restrict__ tc, PsoStateDev s) {
    __shared__ double s_pf[1024];
    __shared__ int s_count;
    const int run = blockIdx.x;
    const int p = threadIdx.x;
    const int P = g.n_particles;
    const int it = s.iter ? s.iter[run] : iter_arg;
    if (p == 0) s_count = 0;
    __syncthreads();
    const int64_t row = (int64_t)run * P + p;
    double x[4];
    if (p < P) {
#pragma unroll
        for (int d = 0; d < 4; ++d) x[d] = s.x[4 * row + d];
        const bool inside = in_box(x);
        const double f = inside ? fitness[row] : -INFINITY;
        double pf = s.pbest_f[row];
        if (f > pf) {
            pf = f;
            s.pbest_f[row] = f;
            s.pbest_tc[row] = tc[row];
#pragma unroll
            for (int d = 0; d < 4; ++d) s.pbest_x[4 * row + d] = x[d];
        }
        s_pf[p] = pf;
        if (inside) atomicAdd(&s_count, 1);
    }
    __syncthreads();
    if (p < P) {
        int best = -1;
        for (int d = -g.n_neighbours; d <= g.n_neighbours; ++d) {
            const int q = ((p + d) % P + P) % P;
            if (best < 0 || s_pf[q] > s_pf[best] || (s_pf[q] == s_pf[best] && q < best)) best = q;
        }
        const int64_t lrow = (int64_t)run * P + best;
        const double w = g.n_iter <= 1 ? g.w_start
                                       : __dadd_rn(g.w_start, __dmul_rn(__dsub_rn(g.w_end, g.w_start),
                                                                        __ddiv_rn((double)it, (double)(g.n_iter - 1))));
        double r1[4], r2[4];
        draw4(g, (uint32_t)run, (uint32_t)it, (uint32_t)p, 0, r1);
        draw4(g, (uint32_t)run, (uint32_t)it, (uint32_t)p, 1, r2);
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const double a = __dmul_rn(w, s.v[4 * row + d]);
            const double b = __dmul_rn(__dmul_rn(g.c1, r1[d]), __dsub_rn(s.pbest_x[4 * row + d], x[d]));
            const double c = __dmul_rn(__dmul_rn(g.c2, r2[d]), __dsub_rn(s.pbest_x[4 * lrow + d], x[d]));
            double vn = __dadd_rn(__dadd_rn(a, b), c);
            vn = fmin(fmax(vn, -g.vmax), g.vmax);
            s.v[4 * row + d] = vn;
            x[d] = __dadd_rn(x[d], vn);
        }
    }
    __syncthreads();   // every thread has read pbest_x of its local best before positions move on
    if (p < P) {
#pragma unroll
        for (int d = 0; d < 4; ++d) s.x[4 * row + d] = x[d];
    }
    if (p == 0) {
        if (s.iter) s.iter[run] = it + 1;
        if (s.evals) s.evals[run] += s_count;
    }
}

__global__ void pso_result_kernel(PsoDev g, PsoStateDev s, fcas_search_result* __restrict__ out) {
    const int run = blockIdx.x * blockDim.x + threadIdx.x;
    if (run >= g.n_runs) return;
    const int P = g.n_particles;
    int best = 0;
    for (int p = 1; p < P; ++p)
        if (s.pbest_f[(int64_t)run * P + p] > s.pbest_f[(int64_t)run * P + best]) best = p;
    const int64_t row = (int64_t)run * P + best;
    fcas_search_result r;
    r.fitness = s.pbest_f[row];
    for (int d = 0; d < 4; ++d) {
        const double lo = g.box[2 * d], hi = g.box[2 * d + 1];
        r.theta[d] = __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), s.pbest_x[4 * row + d]));
    }
    r.tc = s.pbest_tc[row];
    r.evaluations = s.evals ? s.evals[run] : -1;
    out[run] = r;
}

int pso_validate(const fcas_pso_config* cfg, char* msg, size_t len) {
    if (!cfg) return snprintf(msg, len, "NULL PSO configuration"), FCAS_ERR_INVALID;
    if (cfg->n_runs < 1 || cfg->n_particles < 1 || cfg->n_particles > 1024 || cfg->n_iter < 1 ||
        cfg->n_neighbours < 0)
        return snprintf(msg, len, "PSO sizes: need n_runs >= 1, 1 <= n_particles <= 1024, n_iter >= 1, "
                                  "n_neighbours >= 0"),
               FCAS_ERR_INVALID;
    for (int d = 0; d < 4; ++d) {
        const double lo = cfg->box[2 * d], hi = cfg->box[2 * d + 1];
        if (!(std::isfinite(lo) && std::isfinite(hi) && hi > lo))
            return snprintf(msg, len, "PSO box dimension %d: need finite lo < hi", d), FCAS_ERR_INVALID;
    }
    if (!(cfg->box[4] > 0.0 && cfg->box[6] > 0.0))
        return snprintf(msg, len, "PSO box: chirp times must be > 0"), FCAS_ERR_INVALID;
    const double ws[5] = {cfg->w_start, cfg->w_end, cfg->c1, cfg->c2, cfg->vmax};
    for (double w : ws)
        if (!std::isfinite(w)) return snprintf(msg, len, "PSO weights must be finite"), FCAS_ERR_INVALID;
    if (!(cfg->vmax > 0.0)) return snprintf(msg, len, "PSO vmax must be > 0"), FCAS_ERR_INVALID;
    return FCAS_OK;
}

PsoDev pso_dev(const fcas_pso_config* cfg) {
    PsoDev g;
    g.n_runs = cfg->n_runs;
    g.n_particles = cfg->n_particles;
    g.n_iter = cfg->n_iter;
    g.n_neighbours = cfg->n_neighbours;
    g.key0 = (uint32_t)(cfg->seed & 0xFFFFFFFFu);
    g.key1 = (uint32_t)(cfg->seed >> 32);
    for (int d = 0; d < 8; ++d) g.box[d] = cfg->box[d];
    g.w_start = cfg->w_start;
    g.w_end = cfg->w_end;
    g.c1 = cfg->c1;
    g.c2 = cfg->c2;
    g.vmax = cfg->vmax;
    return g;
}

static unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_pso_init(const PsoDev& g, const PsoStateDev& s, cudaStream_t st) {
    pso_init_kernel<<<blocks_for((int64_t)g.n_runs * g.n_particles, 128), 128, 0, st>>>(g, s);
    return cudaGetLastError();
}

cudaError_t launch_pso_theta(const PsoDev& g, const PsoStateDev& s, double* theta, cudaStream_t st) {
    pso_theta_kernel<<<blocks_for((int64_t)g.n_runs * g.n_particles, 128), 128, 0, st>>>(g, s, theta);
    return cudaGetLastError();
}

cudaError_t launch_pso_update(const PsoDev& g, int32_t iter, const double* fitness, const int64_t* tc,
                              const PsoStateDev& s, cudaStream_t st) {
    const int threads = ((g.n_particles + 31) / 32) * 32;
    pso_update_kernel<<<g.n_runs, threads, 0, st>>>(g, iter, fitness, tc, s);
    return cudaGetLastError();
}

cudaError_t launch_pso_result(const PsoDev& g, const PsoStateDev& s, fcas_search_result* out, cudaStream_t st) {
    pso_result_kernel<<<blocks_for(g.n_runs, 64), 64, 0, st>>>(g, s, out);
    return cudaGetLastError();
}

}  // namespace fcas

using namespace fcas;

extern "C" int fcas_pso_init(const fcas_pso_config* cfg, const fcas_pso_state* state, void* stream) {
    char msg[256];
    int rc = pso_validate(cfg, msg, sizeof(msg));
    if (rc) return report_error(rc, msg);
    if (!state || !state->x || !state->v || !state->pbest_x || !state->pbest_f || !state->pbest_tc)
        return report_error(FCAS_ERR_INVALID, "fcas_pso_init: NULL state array");
    PsoStateDev s{state->x, state->v, state->pbest_x, state->pbest_f, state->pbest_tc, nullptr, nullptr};
    cudaError_t e = launch_pso_init(pso_dev(cfg), s, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FCAS_OK : report_error(FCAS_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" int fcas_pso_update(const fcas_pso_config* cfg, int32_t iter, const double* fitness, const int64_t* tc,
                               const fcas_pso_state* state, void* stream) {
    char msg[256];
    int rc = pso_validate(cfg, msg, sizeof(msg));
    if (rc) return report_error(rc, msg);
    if (iter < 0 || iter >= cfg->n_iter) return report_error(FCAS_ERR_INVALID, "fcas_pso_update: iter out of range");
    if (!fitness || !tc || !state || !state->x || !state->v || !state->pbest_x || !state->pbest_f ||
        !state->pbest_tc)
        return report_error(FCAS_ERR_INVALID, "fcas_pso_update: NULL array");
    PsoStateDev s{state->x, state->v, state->pbest_x, state->pbest_f, state->pbest_tc, nullptr, nullptr};
    cudaError_t e = launch_pso_update(pso_dev(cfg), iter, fitness, tc, s, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FCAS_OK : report_error(FCAS_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" int fcas_pso_theta(const fcas_pso_config* cfg, const double* x, double* theta, void* stream) {
    char msg[256];
    int rc = pso_validate(cfg, msg, sizeof(msg));
    if (rc) return report_error(rc, msg);
    if (!x || !theta) return report_error(FCAS_ERR_INVALID, "fcas_pso_theta: NULL array");
    PsoStateDev s{const_cast<double*>(x), nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = launch_pso_theta(pso_dev(cfg), s, theta, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FCAS_OK : report_error(FCAS_ERR_CUDA, cudaGetErrorString(e));
}
