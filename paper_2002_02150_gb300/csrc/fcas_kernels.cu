// Fitness path: per-particle geometry, pass A (fused template x data x delay phase feeding the
// first FFT pass), pass B (second FFT pass + antenna projection + partial argmax over t_c) and
// the final argmax. The length-N inverse transform over t_c is split as N = N1 N2 with
// k = k1 + N1 k2 and t = ta + N2 tb:
//   Z[ta + N2 tb] = sum_k1 e^{2 pi i k1 tb / N1} [ e^{2 pi i k1 ta / N} sum_k2 Q[k1 + N1 k2] e^{2 pi i k2 ta / N2} ]
// Pass A computes the bracket for every column k1 (length-N2 transforms) and stores it as
// A[ta][k1]; pass B transforms every row ta over k1 (length N1).
#include <cfloat>

#include "fcas_fft.cuh"
#include "fcas_kernels.cuh"

namespace fcas {

// ------------------------------------------------------------------------------------------
// Geometry: Sec. II eq. detresponse (U = F(alpha, delta, 0), Delta^i), Sec. II.C/II.D
// (G = sum_i sigma_i^2 U^i U^i^T) and Sec. II.B (chirp times -> phase coefficients).
// ------------------------------------------------------------------------------------------
__global__ void geometry_kernel(const double* __restrict__ theta, int64_t n, ParticleParams* __restrict__ out,
                                const double* __restrict__ det9, const double* __restrict__ s2, int n_det,
                                double f_star, double df) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double alpha = theta[4 * p + 0], delta = theta[4 * p + 1];
    const double tau0 = theta[4 * p + 2], tau15 = theta[4 * p + 3];
    ParticleParams pp;
    for (int q = 0; q < 4; ++q) pp.c[q] = 0.0;
    for (int i = 0; i < FCAS_MAX_DET; ++i) pp.dturn[i] = pp.u[i][0] = pp.u[i][1] = 0.0;
    pp.ginv[0] = pp.ginv[1] = pp.ginv[2] = 0.0;
    pp.chol[0] = pp.chol[1] = pp.chol[2] = 0.0;
    pp.valid = 0;
    pp.pad = 0;
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
    }
    out[p] = pp;
}

cudaError_t launch_geometry(const double* theta, int64_t n, ParticleParams* out, const double* det9,
                            const double* sigma2_scaled, int n_det, double f_star, double df, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int threads = 128;
    const int64_t blocks = (n + threads - 1) / threads;
    geometry_kernel<<<(unsigned)blocks, threads, 0, s>>>(theta, n, out, det9, sigma2_scaled, n_det, f_star, df);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Phase of Q_i[k] = Y_i[k] e^{2 pi i (psi(f_k)/2pi + f_k Delta^i)} (Sec. II.B, eq. data_template_innprod)
// ------------------------------------------------------------------------------------------

// frac((ah + al)(bh + bl)) with the leading product split exactly: the result is the product
// reduced by an integer, accurate to a few float ulps of 1 turn.
__device__ __forceinline__ float frac_mul_ff(float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    return __fadd_rn(__fsub_rn(p, rintf(p)), e);
}

__device__ __forceinline__ float round_nearest(float x) { return rintf(x); }
__device__ __forceinline__ double round_nearest(double x) { return rint(x); }

struct ChirpF {
    float ch[4], cl[4];
    float dh[FCAS_MAX_DET], dl[FCAS_MAX_DET];
};

__device__ __forceinline__ void split_ff(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

__device__ __forceinline__ float chirp_frac(const BasisF& b, const ChirpF& c) {
    float s = frac_mul_ff(c.ch[0], c.cl[0], b.a.x, b.a.y);
    s += frac_mul_ff(c.ch[1], c.cl[1], b.a.z, b.a.w);
    s += frac_mul_ff(c.ch[2], c.cl[2], b.b.x, b.b.y);
    s += frac_mul_ff(c.ch[3], c.cl[3], b.b.z, b.b.w);
    return s - rintf(s);
}

__device__ __forceinline__ double chirp_frac(const BasisD& b, const ParticleParams& pp) {
    double s = pp.c[0] * b.a.x + pp.c[1] * b.a.y + pp.c[2] * b.b.x + pp.c[3] * b.b.y;
    return s - rint(s);
}

__device__ __forceinline__ float2 unit_phasor(float turns) {
    float sn, cs;
    sincospif(2.0f * turns, &sn, &cs);
    return make_float2(cs, sn);
}
__device__ __forceinline__ double2 unit_phasor(double turns) {
    double sn, cs;
    sincospi(2.0 * turns, &sn, &cs);
    return make_double2(cs, sn);
}

// ------------------------------------------------------------------------------------------
// Pass A
// ------------------------------------------------------------------------------------------
template <typename Real, int LOG_L>
__global__ void __launch_bounds__(pass_a_k1b(LOG_L) * ((1 << LOG_L) / pass_a_v(LOG_L)))
pass_a_kernel(const cplx<Real>* __restrict__ y, const Basis<Real>* __restrict__ basis,
              const ParticleParams* __restrict__ params, int64_t p0, int n_det, int log_n1,
              cplx<Real>* __restrict__ out, const cplx<Real>* __restrict__ tw, int tw_shift,
              const cplx<Real>* __restrict__ tw_lo, const cplx<Real>* __restrict__ tw_hi) {
    using C = cplx<Real>;
    constexpr int L = 1 << LOG_L;
    constexpr int V = pass_a_v(LOG_L);
    constexpr int G = L / V;
    constexpr int K1B = pass_a_k1b(LOG_L);
    constexpr int VH = V / 2;    // values with k2 < L/2; the rest of the column is zero (k >= N/2)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);

    const int c = threadIdx.x % K1B;
    const int j = threadIdx.x / K1B;
    const int blk = blockIdx.y;
    const int k1 = blk * K1B + c;
    const int64_t p = blockIdx.x;
    const ParticleParams& pp = params[p0 + p];
    const int64_t n1 = (int64_t)1 << log_n1;
    const int64_t nblk = n1 / K1B;

    Real chirp[VH];
    Real kf[VH];
    ChirpF cf;
    if constexpr (sizeof(Real) == 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r) split_ff(pp.c[r], cf.ch[r], cf.cl[r]);
    }
    const Basis<Real>* bcol = basis + (int64_t)blk * (L / 2) * K1B + c;
#pragma unroll
    for (int q = 0; q < VH; ++q) {
        const int k2 = j + q * G;
        kf[q] = (Real)(k1 + n1 * k2);
        const Basis<Real> b = bcol[(int64_t)k2 * K1B];
        if constexpr (sizeof(Real) == 4) chirp[q] = chirp_frac(b, cf);
        else chirp[q] = chirp_frac(b, pp);
    }

    for (int i = 0; i < n_det; ++i) {
        float dh = 0.f, dl = 0.f;
        if constexpr (sizeof(Real) == 4) split_ff(pp.dturn[i], dh, dl);
        const C* ycol = y + ((int64_t)i * nblk + blk) * (L / 2) * K1B + c;
        C v[V];
#pragma unroll
        for (int q = 0; q < VH; ++q) {
            const C yv = ycol[(int64_t)(j + q * G) * K1B];
            Real th;
            if constexpr (sizeof(Real) == 4) {
                th = chirp[q] + frac_mul_ff(kf[q], 0.0f, dh, dl);
            } else {
                th = chirp[q] + kf[q] * pp.dturn[i];
            }
            th -= round_nearest(th);
            v[q] = cmul(yv, unit_phasor(th));
        }
#pragma unroll
        for (int q = VH; q < V; ++q) v[q] = mkc((Real)0, (Real)0);

        block_fft<Real, +1, LOG_L, V>(v, smem + c, K1B, j, tw, tw_shift);

        C* orow = out + (((int64_t)p * n_det + i) * L) * n1 + k1;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int ta = j + q * G;
            const int m = k1 * ta;   // < N
            const C w = cmul(__ldg(tw_hi + (m >> kTwLoBits)), __ldg(tw_lo + (m & ((1 << kTwLoBits) - 1))));
            orow[(int64_t)ta * n1] = cmul(v[q], w);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Pass B + antenna projection + partial argmax (Sec. II.C: analytic maximisation over A_k)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ bool better(double v, int64_t t, double bv, int64_t bt) {
    return v > bv || (v == bv && t < bt);
}

template <typename Real, int LOG_L>
__global__ void __launch_bounds__(pass_b_tb(LOG_L) * ((1 << LOG_L) / pass_b_v(LOG_L)))
pass_b_kernel(const cplx<Real>* __restrict__ inter, const ParticleParams* __restrict__ params, int64_t p0,
              int n_det, int log_n2, int64_t n_samples, const cplx<Real>* __restrict__ tw, int tw_shift,
              Partial* __restrict__ partials) {
    using C = cplx<Real>;
    constexpr int L = 1 << LOG_L;
    constexpr int V = pass_b_v(LOG_L);
    constexpr int G = L / V;
    constexpr int TB = pass_b_tb(LOG_L);
    constexpr int NT = TB * G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    constexpr int NRED = NT >= 32 ? NT / 32 : NT;
    __shared__ double red_v[NRED];
    __shared__ int64_t red_t[NRED];

    const int j = threadIdx.x % G;
    const int c = threadIdx.x / G;
    const int64_t n2 = (int64_t)1 << log_n2;
    const int64_t ta = (int64_t)blockIdx.x * TB + c;
    const int64_t p = blockIdx.y;
    const ParticleParams& pp = params[p0 + p];

    C w1[V], w2[V];
#pragma unroll
    for (int q = 0; q < V; ++q) w1[q] = w2[q] = mkc((Real)0, (Real)0);

    for (int i = 0; i < n_det; ++i) {
        const C* row = inter + (((int64_t)p * n_det + i) * n2 + ta) * L;
        C v[V];
#pragma unroll
        for (int q = 0; q < V; ++q) v[q] = row[j + q * G];
        block_fft<Real, +1, LOG_L, V>(v, smem + c * L, 1, j, tw, tw_shift);
        const Real up = (Real)pp.u[i][0], ux = (Real)pp.u[i][1];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            w1[q].x += up * v[q].x;
            w1[q].y += up * v[q].y;
            w2[q].x += ux * v[q].x;
            w2[q].y += ux * v[q].y;
        }
    }
    const Real l11 = (Real)pp.chol[0], l21 = (Real)pp.chol[1], l22 = (Real)pp.chol[2];
    double best = -DBL_MAX;
    int64_t bt = INT64_MAX;
#pragma unroll
    for (int q = 0; q < V; ++q) {
        const int64_t t = ta + n2 * (j + q * G);
        // Gamma^2(t) = W^H G^-1 W = |l11 W+ + l21 Wx|^2 + |l22 Wx|^2, W_a = sum_i U_a^i Z_i(t)
        const Real ax = l11 * w1[q].x + l21 * w2[q].x, ay = l11 * w1[q].y + l21 * w2[q].y;
        const Real bx = l22 * w2[q].x, by = l22 * w2[q].y;
        const double gam = (double)(ax * ax + ay * ay + bx * bx + by * by);
        if (t < n_samples && better(gam, t, best, bt)) {
            best = gam;
            bt = t;
        }
    }
    if constexpr (NT >= 32) {
        // NT is a multiple of 32: every warp is full
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, off);
            const int64_t ot = __shfl_down_sync(0xffffffffu, bt, off);
            if (better(ov, ot, best, bt)) { best = ov; bt = ot; }
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { red_v[warp] = best; red_t[warp] = bt; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < NT / 32; ++w)
                if (better(red_v[w], red_t[w], best, bt)) { best = red_v[w]; bt = red_t[w]; }
            partials[p * gridDim.x + blockIdx.x] = Partial{best, bt};
        }
    } else {
        // fewer than 32 threads: no shuffles over lanes that do not exist
        red_v[threadIdx.x] = best;
        red_t[threadIdx.x] = bt;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < NT; ++w)
                if (better(red_v[w], red_t[w], best, bt)) { best = red_v[w]; bt = red_t[w]; }
            partials[p * gridDim.x + blockIdx.x] = Partial{best, bt};
        }
    }
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
// dispatch on the transform lengths
// ------------------------------------------------------------------------------------------
int pass_a_k1b_for(int log_n2) {
    switch (log_n2) {
#define FCAS_CASE(LG) case LG: return pass_a_k1b(LG);
        FCAS_CASE(2) FCAS_CASE(3) FCAS_CASE(4) FCAS_CASE(5) FCAS_CASE(6) FCAS_CASE(7) FCAS_CASE(8)
        FCAS_CASE(9) FCAS_CASE(10) FCAS_CASE(11) FCAS_CASE(12)
#undef FCAS_CASE
        default: return -1;
    }
}

int pass_b_blocks_per_particle(int log_n1, int log_n2) {
    switch (log_n1) {
#define FCAS_CASE(LG) case LG: return (1 << log_n2) / pass_b_tb(LG);
        FCAS_CASE(2) FCAS_CASE(3) FCAS_CASE(4) FCAS_CASE(5) FCAS_CASE(6) FCAS_CASE(7) FCAS_CASE(8)
        FCAS_CASE(9) FCAS_CASE(10) FCAS_CASE(11) FCAS_CASE(12)
#undef FCAS_CASE
        default: return -1;
    }
}

template <typename Real, int LG>
static cudaError_t pass_a_at(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np, void* inter,
                             cudaStream_t s) {
    constexpr int K1B = pass_a_k1b(LG);
    constexpr int THREADS = K1B * ((1 << LG) / pass_a_v(LG));
    const size_t smem = sizeof(cplx<Real>) * (size_t)K1B * (1 << LG);
    auto kern = pass_a_kernel<Real, LG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)np, (unsigned)((1 << pl.log_n1) / K1B));
    kern<<<grid, THREADS, smem, s>>>(static_cast<const cplx<Real>*>(pl.y), static_cast<const Basis<Real>*>(pl.basis),
                                     params, p0, pl.n_det, pl.log_n1, static_cast<cplx<Real>*>(inter),
                                     static_cast<const cplx<Real>*>(pl.tw), pl.tw_shift_a,
                                     static_cast<const cplx<Real>*>(pl.tw_lo), static_cast<const cplx<Real>*>(pl.tw_hi));
    return cudaGetLastError();
}

template <typename Real, int LG>
static cudaError_t pass_b_at(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np,
                             const void* inter, Partial* partials, cudaStream_t s) {
    constexpr int TB = pass_b_tb(LG);
    constexpr int THREADS = TB * ((1 << LG) / pass_b_v(LG));
    const size_t smem = sizeof(cplx<Real>) * (size_t)TB * (1 << LG);
    auto kern = pass_b_kernel<Real, LG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((1 << pl.log_n2) / TB), (unsigned)np);
    kern<<<grid, THREADS, smem, s>>>(static_cast<const cplx<Real>*>(inter), params, p0, pl.n_det, pl.log_n2,
                                     pl.n_samples, static_cast<const cplx<Real>*>(pl.tw), pl.tw_shift_b, partials);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_pass_a(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np, void* inter,
                          cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    switch (pl.log_n2) {
#define FCAS_CASE(LG) case LG: return pass_a_at<Real, LG>(pl, params, p0, np, inter, s);
        FCAS_CASE(2) FCAS_CASE(3) FCAS_CASE(4) FCAS_CASE(5) FCAS_CASE(6) FCAS_CASE(7) FCAS_CASE(8)
        FCAS_CASE(9) FCAS_CASE(10) FCAS_CASE(11) FCAS_CASE(12)
#undef FCAS_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename Real>
cudaError_t launch_pass_b(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np,
                          const void* inter, Partial* partials, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    switch (pl.log_n1) {
#define FCAS_CASE(LG) case LG: return pass_b_at<Real, LG>(pl, params, p0, np, inter, partials, s);
        FCAS_CASE(2) FCAS_CASE(3) FCAS_CASE(4) FCAS_CASE(5) FCAS_CASE(6) FCAS_CASE(7) FCAS_CASE(8)
        FCAS_CASE(9) FCAS_CASE(10) FCAS_CASE(11) FCAS_CASE(12)
#undef FCAS_CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_pass_a<float>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, void*, cudaStream_t);
template cudaError_t launch_pass_a<double>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, void*, cudaStream_t);
template cudaError_t launch_pass_b<float>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, const void*,
                                          Partial*, cudaStream_t);
template cudaError_t launch_pass_b<double>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, const void*,
                                           Partial*, cudaStream_t);

}  // namespace fcas
