// Fitness path, per-particle and host-side parts: geometry, the final argmax, the shape helpers
// of the two passes, the per-stage twiddle tables, and the FP32 / binary64 instantiations of the
// passes (fcas_passes.cuh).
#include "fcas_passes.cuh"

namespace fcas {

// ------------------------------------------------------------------------------------------
// Geometry: Sec. II eq. detresponse (U = F(alpha, delta, 0), Delta^i), Sec. II.C/II.D
// (G = sum_i sigma_i^2 U^i U^i^T) and Sec. II.B (chirp times -> phase coefficients).
// ------------------------------------------------------------------------------------------
__global__ void geometry_kernel(const double* __restrict__ theta, int64_t n, ParticleParams* __restrict__ out,
                                const double* __restrict__ det9, const double* __restrict__ s2, int n_det,
                                double f_star, double df, int64_t kstep) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double alpha = theta[4 * p + 0], delta = theta[4 * p + 1];
    const double tau0 = theta[4 * p + 2], tau15 = theta[4 * p + 3];
    ParticleParams pp;
    for (int q = 0; q < 4; ++q) pp.c[q] = 0.0;
    for (int i = 0; i < FCAS_MAX_DET; ++i) pp.dturn[i] = pp.u[i][0] = pp.u[i][1] = pp.w1[i] = pp.w2[i] = 0.0;
    pp.ginv[0] = pp.ginv[1] = pp.ginv[2] = 0.0;
    pp.chol[0] = pp.chol[1] = pp.chol[2] = 0.0;
    pp.valid = 0;
    pp.taylor_ok = 0;
    const bool ok = isfinite(alpha) && isfinite(delta) && isfinite(tau0) && isfinite(tau15) && tau0 > 0.0 &&
                    tau15 > 0.0;
    if (ok) {
        double sa, ca, sd, cd;
        sincos(alpha, &sa, &ca);
        sincos(delta, &sd, &cd);
        const double nx = cd * ca, ny = cd * sa, nz = sd;
        const double bx[3] = {sa, -ca, 0.0};             // -alpha_hat
        const double by[3] = {-sd * ca, -sd * sa, cd};   // delta_hat
        double g11 = 0.0, g12 = 0.0, g22 = 0.0;
        for (int i = 0; i < n_det; ++i) {
            const double* d = det9 + 9 * i;
            pp.dturn[i] = -(d[0] * nx + d[1] * ny + d[2] * nz) / kCLight * df;
            const double xX = d[3] * bx[0] + d[4] * bx[1] + d[5] * bx[2];
            const double xY = d[3] * by[0] + d[4] * by[1] + d[5] * by[2];
            const double yX = d[6] * bx[0] + d[7] * bx[1] + d[8] * bx[2];
            const double yY = d[6] * by[0] + d[7] * by[1] + d[8] * by[2];
            const double fp = 0.5 * (xX * xX - xY * xY - yX * yX + yY * yY);
            const double fx = xX * xY - yX * yY;
            pp.u[i][0] = fp;
            pp.u[i][1] = fx;
            g11 += s2[i] * fp * fp;
            g12 += s2[i] * fp * fx;
            g22 += s2[i] * fx * fx;
        }
        const double det = g11 * g22 - g12 * g12;
        const double tr = g11 + g22;
        if (det < kRank1Rtol * (0.5 * tr) * (0.5 * tr)) {
            const double lam = 0.5 * tr + sqrt(0.25 * (g11 - g22) * (g11 - g22) + g12 * g12);
            double e1 = lam - g22, e2 = g12;
            double f1 = g12, f2 = lam - g11;
            if (f1 * f1 + f2 * f2 > e1 * e1 + e2 * e2) { e1 = f1; e2 = f2; }
            const double nrm = e1 * e1 + e2 * e2;
            if (lam > 0.0 && nrm > 0.0) {
                pp.ginv[0] = e1 * e1 / nrm / lam;
                pp.ginv[1] = e1 * e2 / nrm / lam;
                pp.ginv[2] = e2 * e2 / nrm / lam;
            }
        } else {
            pp.ginv[0] = g22 / det;
            pp.ginv[1] = -g12 / det;
            pp.ginv[2] = g11 / det;
        }
        // Cholesky factor of G^-1 so that Gamma^2 = |l11 W+ + l21 Wx|^2 + |l22 Wx|^2 is a sum of
        // squares (no cancellation when F is ill-conditioned)
        if (pp.ginv[0] > 0.0) {
            const double l11 = sqrt(pp.ginv[0]);
            const double l21 = pp.ginv[1] / l11;
            pp.chol[0] = l11;
            pp.chol[1] = l21;
            pp.chol[2] = sqrt(fmax(0.0, pp.ginv[2] - l21 * l21));
        } else {
            pp.chol[2] = sqrt(fmax(0.0, pp.ginv[2]));
        }
        for (int i = 0; i < n_det; ++i) {
            pp.w1[i] = pp.chol[0] * pp.u[i][0] + pp.chol[1] * pp.u[i][1];
            pp.w2[i] = pp.chol[2] * pp.u[i][1];
        }
        // (tau0, tau1.5) -> x = pi M f_*, eta; then the 2PN chirp times tau1, tau2.
        const double pi = 0.5 * kTwoPi;
        const double x = 5.0 * tau15 / (32.0 * pi * tau0);
        const double cx = cbrt(x);
        const double eta = 1.0 / (cx * cx) / (8.0 * f_star * tau15);
        const double tau1 = 5.0 / (192.0 * pi * f_star * eta * x) * (743.0 / 336.0 + 11.0 * eta / 4.0);
        const double tau2 = 5.0 / (128.0 * pi * f_star * eta * cx) *
                            (3058673.0 / 1016064.0 + 5429.0 * eta / 1008.0 + 617.0 * eta * eta / 144.0);
        pp.c[0] = 0.6 * f_star * tau0;
        pp.c[1] = f_star * tau1;
        pp.c[2] = -1.5 * f_star * tau15;
        pp.c[3] = 3.0 * f_star * tau2;
        pp.valid = 1;
        // Remainder of psi(k + c) = psi(k) + c psi' + c^2 psi''/2 for c <= C (FP32 pass A, C + 1
        // adjacent columns per lane group, C = 3 or 7): at most C^3/6 max |psi'''| over the band,
        // taken at k_b = f_*/df - 2 (C + 1) (the band's lowest bin, less the C by which an anchor bin
        // may lie below it, with margin), where |psi'''| <= sum_m |c_m| e_m (e_m + 1) (e_m + 2)
        // phi^-e_m / k^3. Bit 0: C = 3; bit 1: C = 7.
        for (int bit = 0; bit < 2; ++bit) {
            const double cm = bit == 0 ? 3.0 : 7.0;
            const double kb = f_star / df - 2.0 * (cm + 1.0);
            if (kb < 1.0) continue;
            const double r = f_star / (kb * df);   // phi^-1 at k_b
            const double r13 = cbrt(r);
            const double d3 = (fabs(pp.c[0]) * (440.0 / 27.0) * r * r13 * r13 + fabs(pp.c[1]) * 6.0 * r +
                               fabs(pp.c[2]) * (80.0 / 27.0) * r13 * r13 + fabs(pp.c[3]) * (28.0 / 27.0) * r13) /
                              (kb * kb * kb);
            if (cm * cm * cm / 6.0 * d3 < 1e-7) pp.taylor_ok |= 1 << bit;
        }
    }
    for (int r = 0; r < 4; ++r) {
        pp.ch[r] = (float)pp.c[r];
        pp.cl[r] = (float)(pp.c[r] - (double)pp.ch[r]);
    }
    for (int i = 0; i < FCAS_MAX_DET; ++i) {
        if (i >= n_det) pp.w1[i] = pp.w2[i] = 0.0;
        pp.dh[i] = (float)pp.dturn[i];
        pp.dl[i] = (float)(pp.dturn[i] - (double)pp.dh[i]);
        pp.w1f[i] = (float)pp.w1[i];
        pp.w2f[i] = (float)pp.w2[i];
        double u = (double)kstep * pp.dturn[i];   // |u| < 2^24 turns, exact to ~1e-9
        u -= rint(u);
        double su, cu;
        sincospi(2.0 * u, &su, &cu);
        pp.dstep[i] = make_float2((float)cu, (float)su);
    }
    out[p] = pp;
}

cudaError_t launch_geometry(const double* theta, int64_t n, ParticleParams* out, const double* det9,
                            const double* sigma2_scaled, int n_det, double f_star, double df, int64_t kstep,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int threads = 128;
    const int64_t blocks = (n + threads - 1) / threads;
    geometry_kernel<<<(unsigned)blocks, threads, 0, s>>>(theta, n, out, det9, sigma2_scaled, n_det, f_star, df,
                                                          kstep);
    return cudaGetLastError();
}

__device__ __forceinline__ bool better(double v, int64_t t, double bv, int64_t bt) {
    return v > bv || (v == bv && t < bt);
}


__global__ void reduce_kernel(const Partial* __restrict__ partials, int64_t nb, const ParticleParams* __restrict__ params,
                              int64_t p0, double* __restrict__ fitness, int64_t* __restrict__ tc) {
    __shared__ double sv[32];
    __shared__ int64_t st[32];
    const int64_t p = blockIdx.x;
    double best = -DBL_MAX;
    int64_t bt = INT64_MAX;
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
        const Partial q = partials[p * nb + b];
        if (better(q.val, q.t, best, bt)) { best = q.val; bt = q.t; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, off);
        const int64_t ot = __shfl_down_sync(0xffffffffu, bt, off);
        if (better(ov, ot, best, bt)) { best = ov; bt = ot; }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sv[warp] = best; st[warp] = bt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x + 31) / 32; ++w)
            if (better(sv[w], st[w], best, bt)) { best = sv[w]; bt = st[w]; }
        const bool ok = params[p0 + p].valid != 0;
        fitness[p0 + p] = ok ? best : __longlong_as_double(0x7ff8000000000000LL);
        tc[p0 + p] = ok ? bt : -1;
    }
}

cudaError_t launch_reduce(const Partial* partials, int64_t nb, const ParticleParams* params, int64_t p0, int64_t np,
                          double* fitness, int64_t* tc, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    reduce_kernel<<<(unsigned)np, 256, 0, s>>>(partials, nb, params, p0, fitness, tc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// shape helpers of the passes
// ------------------------------------------------------------------------------------------
int pass_a_k1b_for(int log_n2, int precision) {
    const int rb = precision == FCAS_PREC_FP32 ? 4 : 8;
    switch (log_n2) {
#define FCAS_CASE(LG) case LG: return pass_a_k1b(LG, rb);
        FCAS_LOG_CASES(FCAS_CASE)
#undef FCAS_CASE
        default: return -1;
    }
}

int pass_b_blocks_per_particle(int log_n1, int log_n2, int precision) {
    const bool fp32 = precision == FCAS_PREC_FP32;
    switch (log_n1) {
#define FCAS_CASE(LG) case LG: return (1 << log_n2) / pass_b_tb(LG, fp32 ? 4 : 8);
        FCAS_LOG_CASES(FCAS_CASE)
#undef FCAS_CASE
        default: return -1;
    }
}

bool pass_a_radix8_available(int log_n2, int precision, int k1b) {
    if (precision == FCAS_PREC_FP32) return log_n2 >= 10 && ((log_n2 <= 11 && k1b == 4) || (log_n2 <= 12 && k1b == 2));
    return log_n2 >= 10 && log_n2 <= 12 && precision == FCAS_PREC_FF && k1b == 2;
}

int pass_a_default_radix_bits(int log_n2, int precision) {
    // float-float: radix 8 halves the registers per thread (16 resident warps per SM instead of 8)
    return precision == FCAS_PREC_FF && log_n2 == 11 ? 3 : 4;
}

int pass_a_k1b_variants(int log_n2, int precision, int* out) {
    const int rb = precision == FCAS_PREC_FP32 ? 4 : 8;
    int n = 0;
    switch (log_n2) {
#define FCAS_CASE(LG)                                                                       \
    case LG: {                                                                              \
        const int kd = pass_a_k1b(LG, rb);                                                  \
        out[n++] = kd;                                                                      \
        if (rb == 4 && LG >= 8) {                                                           \
            if (x2_k1b_ok<LG>(kd / 2)) out[n++] = kd / 2;                                   \
            if (x2_k1b_ok<LG>(kd * 2)) out[n++] = kd * 2;                                   \
            if (LG >= 10 && kd / 2 > 1) out[n++] = 1;                                       \
        }                                                                                   \
        return n;                                                                           \
    }
        FCAS_LOG_CASES(FCAS_CASE)
#undef FCAS_CASE
        default: return 0;
    }
}

template cudaError_t launch_pass_a<float>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, void*, cudaStream_t);
template cudaError_t launch_pass_a<double>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, void*, cudaStream_t);
template cudaError_t launch_pass_b<float>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, const void*,
                                          Partial*, cudaStream_t);
template cudaError_t launch_pass_b<double>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, const void*,
                                           Partial*, cudaStream_t);

// ------------------------------------------------------------------------------------------
// per-stage twiddle tables of the radix-16 transforms (create time)
// ------------------------------------------------------------------------------------------
__global__ void stage_table_kernel(int log_l, int maxrb, double2* t64, float2* t32) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = 1 << log_l;
    if (m >= l) return;
    double2 val = make_double2(1.0, 0.0);
    // find the stage that owns entry m: (Ns - 1) <= m < Ns R - 1
    for (int done = 0; done < log_l; done += fftr_radix_bits(log_l, done, maxrb)) {
        const int ns = 1 << done;
        const int r_ = 1 << fftr_radix_bits(log_l, done, maxrb);
        if (ns > 1 && m >= ns - 1 && m < ns * r_ - 1) {
            const int off = m - (ns - 1);
            const int r = off / ns + 1;
            const int jm = off % ns;
            double sn, cs;
            // e^{2 pi i r jm / (Ns R)}, argument reduced exactly before sincospi
            const long long num = ((long long)r * jm) % ((long long)ns * r_);
            sincospi(2.0 * (double)num / (double)(ns * r_), &sn, &cs);
            val = make_double2(cs, sn);
        }
    }
    t64[m] = val;
    t32[m] = make_float2((float)val.x, (float)val.y);
}

unsigned int take_index_checks(cudaStream_t s) {
#ifdef FCAS_CHECKED
    unsigned int h = 0, zero = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) return 0;
    cudaMemcpyFromSymbol(&h, g_index_checks, sizeof(h));
    cudaMemcpyToSymbol(g_index_checks, &zero, sizeof(zero));
    return h;
#else
    (void)s;
    return 0;
#endif
}

cudaError_t launch_stage_tables(int log_l, int maxrb, double2* t64, float2* t32, cudaStream_t s) {
    const int l = 1 << log_l;
    stage_table_kernel<<<(l + 255) / 256, 256, 0, s>>>(log_l, maxrb, t64, t32);
    return cudaGetLastError();
}

}  // namespace fcas
