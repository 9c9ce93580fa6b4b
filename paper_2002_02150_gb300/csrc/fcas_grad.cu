// Adjoint of the coherent fitness at a fixed t_c (envelope theorem): d Gamma^2(theta, t*) / d theta
// for theta = (alpha, delta, tau0, tau1.5) at the argmax t* of a previous fitness evaluation.
//
// With Z_i = sum_k Q_i[k] e^{2 pi i k t*/N}, W = sum_i U^i Z_i and Gamma^2 = Re(W^H G^-1 W) (Sec. II.C),
//   d Gamma^2 = 2 Re(dW^H G^-1 W) - W^H (G^-1 dG G^-1) W,   dW = sum_i (dU^i Z_i + U^i dZ_i),
//   dG = sum_i sigma_i^2 (dU^i U^iT + U^i dU^iT),
// and, since Q_i[k] carries the phase 2 pi (psi(f_k)/2pi + k Delta^i df) (Sec. II.B, II.D),
//   dZ_i/d(alpha, delta) = 2 pi i (d(Delta^i df)/d(alpha, delta)) sum_k k Q_i e^{...},
//   dZ_i/d(tau0, tau1.5) = 2 pi i sum_j (dc_j/dtau) sum_k B_j(k) Q_i e^{...}
// with B_j = phi^-5/3, phi^-1, phi^-2/3, phi^-1/3. A reduction kernel forms the six sums per
// (particle, detector) in one sweep of the band; a per-particle kernel combines them in binary64.
#include <cmath>

#include "fcas_kernels.cuh"

namespace fcas {

constexpr int kGradSums = 12;   // Z, F (= sum k Q), S_53, S_1, S_23, S_13: complex, as (re, im) doubles

template <typename Real>
__global__ void __launch_bounds__(256)
grad_sums_kernel(const cplx<Real>* __restrict__ y, bool y_ff, const Basis<Real>* __restrict__ basis,
                 const ParticleParams* __restrict__ params, const int64_t* __restrict__ tc, int n_det, int log_n,
                 int log_n1, int log_n2, int k1b, int64_t k_lo, int64_t k_hi, double* __restrict__ sums) {
    __shared__ double red[kGradSums][8];
    const int64_t p = blockIdx.x;
    const int i = blockIdx.y;
    const ParticleParams& pp = params[p];
    const int64_t t = tc[p];
    const int64_t n = (int64_t)1 << log_n, n1 = (int64_t)1 << log_n1, half2 = ((int64_t)1 << log_n2) / 2;
    const int64_t per_blk = half2 * k1b;
    double acc[kGradSums];
#pragma unroll
    for (int q = 0; q < kGradSums; ++q) acc[q] = 0.0;
    if (pp.valid && t >= 0) {
        for (int64_t g = threadIdx.x; g < n / 2; g += blockDim.x) {
            const int64_t blk = g / per_blk, rem = g % per_blk;
            const int64_t k = blk * k1b + rem % k1b + n1 * (rem / k1b);
            if (k < k_lo || k > k_hi) continue;
            cplx<Real> yv;
            if constexpr (sizeof(Real) == 8) {
                if (y_ff) {   // float-float layout (FCAS_PREC_FF contexts): 16-byte entries hi/lo re, hi/lo im
                    const float4 q = reinterpret_cast<const float4*>(y)[(blk * n_det + i) * per_blk + rem];
                    yv = make_double2((double)q.x + (double)q.y, (double)q.z + (double)q.w);
                } else {
                    yv = y[(blk * n_det + i) * per_blk + rem];
                }
            } else {
                yv = y[(blk * n_det + i) * per_blk + rem];
            }
            const Basis<Real> b = basis[g];
            const double shift = (double)((k * t) & (n - 1)) / (double)n;   // k t / N mod 1, exact
            double qr, qi, b53, b1, b23, b13;
            if constexpr (sizeof(Real) == 4) {
                const ChirpPowers cpw = chirp_powers(b);
                float s = frac_mul_ff(pp.ch[0], pp.cl[0], cpw.b53.x, cpw.b53.y);
                s += frac_mul_ff(pp.ch[1], pp.cl[1], cpw.b1.x, cpw.b1.y);
                s += frac_mul_ff(pp.ch[2], pp.cl[2], cpw.b23.x, cpw.b23.y);
                s += frac_mul_ff(pp.ch[3], pp.cl[3], cpw.b13.x, cpw.b13.y);
                float th = s + frac_mul_ff((float)k, 0.0f, pp.dh[i], pp.dl[i]) + (float)shift;
                th -= rintf(th);
                float sn, cs;
                sincospif(2.0f * th, &sn, &cs);
                qr = (double)(yv.x * cs - yv.y * sn);
                qi = (double)(yv.x * sn + yv.y * cs);
                b53 = (double)cpw.b53.x + (double)cpw.b53.y;
                b1 = (double)cpw.b1.x + (double)cpw.b1.y;
                b23 = (double)cpw.b23.x + (double)cpw.b23.y;
                b13 = (double)cpw.b13.x + (double)cpw.b13.y;
            } else {
                double th = pp.c[0] * b.a.x + pp.c[1] * b.a.y + pp.c[2] * b.b.x + pp.c[3] * b.b.y;
                th -= rint(th);
                double kd = (double)k * pp.dturn[i];
                th += kd - rint(kd) + shift;
                th -= rint(th);
                double sn, cs;
                sincospi(2.0 * th, &sn, &cs);
                qr = yv.x * cs - yv.y * sn;
                qi = yv.x * sn + yv.y * cs;
                b53 = b.a.x;
                b1 = b.a.y;
                b23 = b.b.x;
                b13 = b.b.y;
            }
            const double kk = (double)k;
            acc[0] += qr;
            acc[1] += qi;
            acc[2] += kk * qr;
            acc[3] += kk * qi;
            acc[4] += b53 * qr;
            acc[5] += b53 * qi;
            acc[6] += b1 * qr;
            acc[7] += b1 * qi;
            acc[8] += b23 * qr;
            acc[9] += b23 * qi;
            acc[10] += b13 * qr;
            acc[11] += b13 * qi;
        }
    }
    // fixed-order reduction: warp shuffles, then the 8 warp partials in order
#pragma unroll
    for (int q = 0; q < kGradSums; ++q) {
        double v = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < kGradSums) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
        sums[(p * n_det + i) * kGradSums + threadIdx.x] = v;
    }
}

// forward-mode dual number for the chirp-coefficient derivatives
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
__device__ __forceinline__ Dual dpow(Dual a, double e) {
    const double pv = pow(a.v, e);
    return {pv, e * pow(a.v, e - 1.0) * a.d};
}

// c_j(tau0, tau1.5) (turns) with derivative along (dt0, dt15), as in the geometry kernel
__device__ void chirp_coeffs_dual(double tau0, double tau15, double dt0, double dt15, double f_star, Dual c[4]) {
    const double pi = 3.14159265358979323846;
    const Dual t0{tau0, dt0}, t15{tau15, dt15};
    const Dual x = (5.0 / (32.0 * pi)) * (t15 / t0);
    const Dual eta = dpow(x, -2.0 / 3.0) / ((8.0 * f_star) * t15);
    const Dual one{1.0, 0.0};
    const Dual tau1 = (5.0 / (192.0 * pi * f_star)) * ((Dual{743.0 / 336.0, 0.0} + (11.0 / 4.0) * eta) / (eta * x));
    const Dual tau2 = (5.0 / (128.0 * pi * f_star)) *
                      ((Dual{3058673.0 / 1016064.0, 0.0} + (5429.0 / 1008.0) * eta + (617.0 / 144.0) * (eta * eta)) /
                       (eta * dpow(x, 1.0 / 3.0)));
    (void)one;
    c[0] = (0.6 * f_star) * t0;
    c[1] = f_star * tau1;
    c[2] = (-1.5 * f_star) * t15;
    c[3] = (3.0 * f_star) * tau2;
}

__global__ void grad_final_kernel(const double* __restrict__ theta, const int64_t* __restrict__ tc, int64_t n,
                                  const double* __restrict__ sums, const double* __restrict__ det9,
                                  const double* __restrict__ s2, int n_det, double f_star, double df,
                                  double* __restrict__ grad) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const double alpha = theta[4 * p], delta = theta[4 * p + 1], tau0 = theta[4 * p + 2], tau15 = theta[4 * p + 3];
    for (int m = 0; m < 4; ++m) grad[4 * p + m] = nan;
    if (!(isfinite(alpha) && isfinite(delta) && tau0 > 0.0 && tau15 > 0.0 && tc[p] >= 0)) return;
    const double two_pi = 6.283185307179586476925286766559;
    double sa, ca, sd, cd;
    sincos(alpha, &sa, &ca);
    sincos(delta, &sd, &cd);
    // basis vectors and their derivatives: [0] value, [1] d/d alpha, [2] d/d delta
    const double nv[3][3] = {{cd * ca, cd * sa, sd}, {-cd * sa, cd * ca, 0.0}, {-sd * ca, -sd * sa, cd}};
    const double bx[3][3] = {{sa, -ca, 0.0}, {ca, sa, 0.0}, {0.0, 0.0, 0.0}};
    const double by[3][3] = {{-sd * ca, -sd * sa, cd}, {sd * sa, -sd * ca, 0.0}, {-cd * ca, -cd * sa, -sd}};
    double u[FCAS_MAX_DET][3][2];    // U^i and its alpha / delta derivatives
    double dd[FCAS_MAX_DET][3];      // delay in turns per bin and its derivatives
    double G[3][3] = {};             // G entries (11, 12, 22) and derivatives
    for (int i = 0; i < n_det; ++i) {
        const double* dv = det9 + 9 * i;
        auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
        const double xX = dot(dv + 3, bx[0]), xY = dot(dv + 3, by[0]), yX = dot(dv + 6, bx[0]), yY = dot(dv + 6, by[0]);
        u[i][0][0] = 0.5 * (xX * xX - xY * xY - yX * yX + yY * yY);
        u[i][0][1] = xX * xY - yX * yY;
        for (int m = 1; m < 3; ++m) {
            const double dxX = dot(dv + 3, bx[m]), dxY = dot(dv + 3, by[m]), dyX = dot(dv + 6, bx[m]),
                         dyY = dot(dv + 6, by[m]);
            u[i][m][0] = xX * dxX - xY * dxY - yX * dyX + yY * dyY;
            u[i][m][1] = dxX * xY + xX * dxY - dyX * yY - yX * dyY;
        }
        for (int m = 0; m < 3; ++m) dd[i][m] = -dot(dv, nv[m]) / kCLight * df;
        for (int m = 0; m < 3; ++m) {
            // m = 0: G itself; m = 1, 2: dG = sum s2 (dU U^T + U dU^T)
            if (m == 0) {
                G[0][0] += s2[i] * u[i][0][0] * u[i][0][0];
                G[0][1] += s2[i] * u[i][0][0] * u[i][0][1];
                G[0][2] += s2[i] * u[i][0][1] * u[i][0][1];
            } else {
                G[m][0] += s2[i] * 2.0 * u[i][m][0] * u[i][0][0];
                G[m][1] += s2[i] * (u[i][m][0] * u[i][0][1] + u[i][0][0] * u[i][m][1]);
                G[m][2] += s2[i] * 2.0 * u[i][m][1] * u[i][0][1];
            }
        }
    }
    const double det = G[0][0] * G[0][2] - G[0][1] * G[0][1];
    const double tr = G[0][0] + G[0][2];
    if (det < kRank1Rtol * (0.5 * tr) * (0.5 * tr)) return;   // rank-1 branch: no gradient (NaN)
    const double gi[3] = {G[0][2] / det, -G[0][1] / det, G[0][0] / det};
    // Z_i, F_i, S_ij
    const double* sp = sums + p * n_det * 12;
    double Wr[2] = {0, 0}, Wi[2] = {0, 0};
    for (int i = 0; i < n_det; ++i)
        for (int a = 0; a < 2; ++a) {
            Wr[a] += u[i][0][a] * sp[12 * i + 0];
            Wi[a] += u[i][0][a] * sp[12 * i + 1];
        }
    auto quad_re = [&](const double* ar, const double* ai, const double* br, const double* bi, const double* g) {
        // Re(a^H Ginv b) with Ginv = [[g0, g1], [g1, g2]]
        const double r0 = g[0] * br[0] + g[1] * br[1], r1 = g[1] * br[0] + g[2] * br[1];
        const double i0 = g[0] * bi[0] + g[1] * bi[1], i1 = g[1] * bi[0] + g[2] * bi[1];
        return ar[0] * r0 + ar[1] * r1 + ai[0] * i0 + ai[1] * i1;
    };
    Dual c0[4], c1[4];
    chirp_coeffs_dual(tau0, tau15, 1.0, 0.0, f_star, c0);
    chirp_coeffs_dual(tau0, tau15, 0.0, 1.0, f_star, c1);
    for (int m = 0; m < 4; ++m) {
        double dWr[2] = {0, 0}, dWi[2] = {0, 0};
        for (int i = 0; i < n_det; ++i) {
            const double* s = sp + 12 * i;
            // dZ_i = 2 pi i * X_i, X_i = (dd_i) F_i or sum_j dc_j S_ij
            double xr, xi;
            if (m < 2) {
                xr = dd[i][m + 1] * s[2];
                xi = dd[i][m + 1] * s[3];
            } else {
                const Dual* c = m == 2 ? c0 : c1;
                xr = c[0].d * s[4] + c[1].d * s[6] + c[2].d * s[8] + c[3].d * s[10];
                xi = c[0].d * s[5] + c[1].d * s[7] + c[2].d * s[9] + c[3].d * s[11];
            }
            const double dzr = -two_pi * xi, dzi = two_pi * xr;
            for (int a = 0; a < 2; ++a) {
                dWr[a] += u[i][0][a] * dzr;
                dWi[a] += u[i][0][a] * dzi;
                if (m < 2) {
                    dWr[a] += u[i][m + 1][a] * s[0];
                    dWi[a] += u[i][m + 1][a] * s[1];
                }
            }
        }
        double gsum = 2.0 * quad_re(dWr, dWi, Wr, Wi, gi);
        if (m < 2) {
            // - W^H Ginv dG Ginv W: Ginv W first, then the dG quadratic form
            const double ar[2] = {gi[0] * Wr[0] + gi[1] * Wr[1], gi[1] * Wr[0] + gi[2] * Wr[1]};
            const double ai[2] = {gi[0] * Wi[0] + gi[1] * Wi[1], gi[1] * Wi[0] + gi[2] * Wi[1]};
            gsum -= quad_re(ar, ai, ar, ai, G[m + 1]);
        }
        grad[4 * p + m] = gsum;
    }
}

template <typename Real>
cudaError_t launch_grad_sums(const FitnessPlan& pl, int k1b, int64_t k_lo, int64_t k_hi, const ParticleParams* params,
                             const int64_t* tc, int64_t n, double* sums, cudaStream_t s, bool y_ff) {
    if (n <= 0) return cudaSuccess;
    dim3 grid((unsigned)n, (unsigned)pl.n_det);
    grad_sums_kernel<Real><<<grid, 256, 0, s>>>(static_cast<const cplx<Real>*>(pl.y), y_ff,
                                                static_cast<const Basis<Real>*>(pl.basis), params, tc, pl.n_det,
                                                pl.log_n, pl.log_n1, pl.log_n2, k1b, k_lo, k_hi, sums);
    return cudaGetLastError();
}

cudaError_t launch_grad_final(const double* theta, const int64_t* tc, int64_t n, const double* sums,
                              const double* det9, const double* s2, int n_det, double f_star, double df, double* grad,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    grad_final_kernel<<<(unsigned)((n + 63) / 64), 64, 0, s>>>(theta, tc, n, sums, det9, s2, n_det, f_star, df, grad);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Gradient polishing: ascent steps along the adjoint gradient, each halved until the fitness
// increases (the differentiation form's use of the adjoint; the paper itself only runs the swarm).
// Per particle, with s = scales (1, 1, tau0, tau1.5) (absolute for the angles, relative for the
// chirp times): direction d = s^2 g / |s g| (a step of length |s| in the metric of s, uphill),
// first trial step length 1, halved after every trial that does not raise the fitness.
// ------------------------------------------------------------------------------------------
__global__ void polish_direction_kernel(const double* __restrict__ theta, const double* __restrict__ grad,
                                        PolishScales sc, int64_t n, double* __restrict__ dir,
                                        double* __restrict__ step, int32_t* __restrict__ done) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double sg[4], norm2 = 0.0;
    bool finite = true;
    for (int m = 0; m < 4; ++m) {
        const double s = sc.s[m] * (m < 2 ? 1.0 : theta[4 * p + m]);
        const double g = grad[4 * p + m];
        finite = finite && isfinite(g) && isfinite(s);
        sg[m] = s * g;
        dir[4 * p + m] = s * s * g;
        norm2 += sg[m] * sg[m];
    }
    const double norm = sqrt(norm2);
    const bool ok = finite && norm > 0.0;
    for (int m = 0; m < 4; ++m) dir[4 * p + m] = ok ? dir[4 * p + m] / norm : 0.0;
    step[p] = 1.0;
    done[p] = ok ? 0 : 1;
}

// the trial point of every particle still searching; NaN (not evaluated) for the others
__global__ void polish_candidate_kernel(const double* __restrict__ theta, const double* __restrict__ dir,
                                        const double* __restrict__ step, const int32_t* __restrict__ done, int64_t n,
                                        double* __restrict__ cand) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    for (int m = 0; m < 4; ++m)
        cand[4 * p + m] = done[p] ? __longlong_as_double(0x7ff8000000000000LL)
                                  : theta[4 * p + m] + step[p] * dir[4 * p + m];
}

// accept a trial that raises the fitness (a NaN trial never does); otherwise halve the step and count
// the particle as still searching
__global__ void polish_accept_kernel(double* __restrict__ theta, double* __restrict__ fit, int64_t* __restrict__ tc,
                                     const double* __restrict__ cand, const double* __restrict__ cfit,
                                     const int64_t* __restrict__ ctc, double* __restrict__ step,
                                     int32_t* __restrict__ done, int32_t* __restrict__ accepted, int64_t n,
                                     int32_t* __restrict__ searching) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || done[p]) return;
    if (cfit[p] > fit[p]) {
        for (int m = 0; m < 4; ++m) theta[4 * p + m] = cand[4 * p + m];
        fit[p] = cfit[p];
        tc[p] = ctc[p];
        accepted[p] += 1;
        done[p] = 1;
    } else {
        step[p] *= 0.5;
        atomicAdd(searching, 1);
    }
}

cudaError_t launch_polish_direction(const double* theta, const double* grad, const PolishScales& sc, int64_t n,
                                    double* dir, double* step, int32_t* done, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    polish_direction_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(theta, grad, sc, n, dir, step, done);
    return cudaGetLastError();
}

cudaError_t launch_polish_candidate(const double* theta, const double* dir, const double* step, const int32_t* done,
                                    int64_t n, double* cand, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    polish_candidate_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(theta, dir, step, done, n, cand);
    return cudaGetLastError();
}

cudaError_t launch_polish_accept(double* theta, double* fit, int64_t* tc, const double* cand, const double* cfit,
                                 const int64_t* ctc, double* step, int32_t* done, int32_t* accepted, int64_t n,
                                 int32_t* searching, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    polish_accept_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(theta, fit, tc, cand, cfit, ctc, step, done,
                                                                     accepted, n, searching);
    return cudaGetLastError();
}

template cudaError_t launch_grad_sums<float>(const FitnessPlan&, int, int64_t, int64_t, const ParticleParams*,
                                             const int64_t*, int64_t, double*, cudaStream_t, bool);
template cudaError_t launch_grad_sums<double>(const FitnessPlan&, int, int64_t, int64_t, const ParticleParams*,
                                              const int64_t*, int64_t, double*, cudaStream_t, bool);

}  // namespace fcas
