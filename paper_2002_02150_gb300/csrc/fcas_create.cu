// Create path (Sec. II.D): twiddle tables, input checks, template norms <h_c|h_c>^i, forward FFT
// of the data in binary64, over-whitening and the re-laid-out band spectrum Y consumed by pass A.
#include "fcas_fft.cuh"
#include "fcas_kernels.cuh"

namespace fcas {

// ------------------------------------------------------------------------------------------
// twiddle tables (binary64 sincospi, rounded once for the FP32 copies)
// ------------------------------------------------------------------------------------------
__global__ void tables_kernel(int log_tw, int log_n, double2* tw64, double2* twlo64, double2* twhi64, float2* tw32,
                              float2* twlo32, float2* twhi32) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ntw = (int64_t)1 << log_tw;
    const int64_t nlo = (int64_t)1 << kTwLoBits;
    const int64_t nhi = log_n > kTwLoBits ? ((int64_t)1 << (log_n - kTwLoBits)) : 1;
    double s, c;
    if (m < ntw) {
        sincospi(2.0 * (double)m / (double)ntw, &s, &c);
        tw64[m] = make_double2(c, s);
        tw32[m] = make_float2((float)c, (float)s);
    }
    if (m < nlo) {
        // e^{2 pi i m / N}: reduce m mod N first so the argument stays in [0, 2)
        const int64_t n = (int64_t)1 << log_n;
        sincospi(2.0 * (double)(m & (n - 1)) / (double)n, &s, &c);
        twlo64[m] = make_double2(c, s);
        twlo32[m] = make_float2((float)c, (float)s);
    }
    if (m < nhi) {
        const int64_t n = (int64_t)1 << log_n;
        sincospi(2.0 * (double)((m << kTwLoBits) & (n - 1)) / (double)n, &s, &c);
        twhi64[m] = make_double2(c, s);
        twhi32[m] = make_float2((float)c, (float)s);
    }
}

cudaError_t launch_tables(int log_n, int log_n1, int log_n2, double2* tw64, double2* twlo64, double2* twhi64,
                          float2* tw32, float2* twlo32, float2* twhi32, cudaStream_t s) {
    const int log_tw = log_n1 > log_n2 ? log_n1 : log_n2;
    int64_t total = (int64_t)1 << log_tw;
    if (total < ((int64_t)1 << kTwLoBits)) total = (int64_t)1 << kTwLoBits;
    const int64_t nhi = log_n > kTwLoBits ? ((int64_t)1 << (log_n - kTwLoBits)) : 1;
    if (total < nhi) total = nhi;
    tables_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(log_tw, log_n, tw64, twlo64, twhi64, tw32, twlo32,
                                                                 twhi32);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// input checks
// ------------------------------------------------------------------------------------------
__global__ void check_finite_kernel(const double* __restrict__ x, int64_t n, int* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) atomicOr(flag, 1);
}

// Circular time shift of each detector's series within its n samples: y_i[t] = x_i[(t - s_i) mod n]
// (shifts already reduced to 0..n-1). Background realisations of Sec. V.
__global__ void time_shift_kernel(const double* __restrict__ x, double* __restrict__ y, int n_det, int64_t n,
                                  DetShifts sh) {
    const int64_t total = (int64_t)n_det * n;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / n);
        const int64_t t = g - (int64_t)i * n;
        int64_t src = t - sh.s[i];
        if (src < 0) src += n;
        y[g] = x[(int64_t)i * n + src];
    }
}

cudaError_t launch_time_shift(const double* x, double* y, int n_det, int64_t n, const DetShifts& sh, cudaStream_t s) {
    const int64_t total = (int64_t)n_det * n;
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    time_shift_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, y, n_det, n, sh);
    return cudaGetLastError();
}

__global__ void split_ff_kernel(const double2* __restrict__ src, float4* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        const float xh = (float)v.x, yh = (float)v.y;
        dst[i] = make_float4(xh, (float)(v.x - (double)xh), yh, (float)(v.y - (double)yh));
    }
}

__global__ void phase_table_ff_kernel(float4* __restrict__ dst, int n) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)m / (double)n, &sn, &cs);
        const float xh = (float)cs, yh = (float)sn;
        dst[m] = make_float4(xh, (float)(cs - (double)xh), yh, (float)(sn - (double)yh));
    }
}

cudaError_t launch_phase_table_ff(void* dst, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    phase_table_ff_kernel<<<(n + 255) / 256, 256, 0, s>>>(static_cast<float4*>(dst), n);
    return cudaGetLastError();
}

cudaError_t launch_split_ff(const double2* src, void* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    split_ff_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, static_cast<float4*>(dst), n);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    check_finite_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, n, flag);
    return cudaGetLastError();
}

__global__ void check_psd_kernel(const double* __restrict__ psd, int n_det, int64_t row, int64_t k_lo, int64_t k_hi,
                                 int* flag) {
    const int64_t nb = k_hi - k_lo + 1;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nb * n_det;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / nb);
        const double v = psd[i * row + k_lo + g % nb];
        if (!(isfinite(v) && v > 0.0)) atomicOr(flag, 2);
    }
}

cudaError_t launch_check_psd(const double* psd, int n_det, int64_t row, int64_t k_lo, int64_t k_hi, int* flag,
                             cudaStream_t s) {
    check_psd_kernel<<<1024, 256, 0, s>>>(psd, n_det, row, k_lo, k_hi, flag);
    return cudaGetLastError();
}

// One-sided noise PSD of every detector from the analytic fit to the aLIGO design sensitivity
// (Sec. II.A noise model; the paper's own curves are not tabulated):
//   S(f) = 1e-49 [x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4/2) / (1 + x^2/2)],  x = f / 215 Hz,
// on the band bins f_k = k df, k_lo <= k <= k_hi, of rows of length `row`; the other bins are set
// to zero (they are never read).
__global__ void analytic_psd_kernel(double* __restrict__ psd, int n_det, int64_t row, int64_t k_lo, int64_t k_hi,
                                    double df) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < row * n_det;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = g % row;
        double v = 0.0;
        if (k >= k_lo && k <= k_hi) {
            const double x = (double)k * df / 215.0;
            const double x2 = x * x;
            v = 1e-49 * (pow(x, -4.14) - 5.0 / x2 + 111.0 * (1.0 - x2 + 0.5 * x2 * x2) / (1.0 + 0.5 * x2));
        }
        psd[g] = v;
    }
}

cudaError_t launch_analytic_psd(double* psd, int n_det, int64_t row, int64_t k_lo, int64_t k_hi, double df,
                                cudaStream_t s) {
    analytic_psd_kernel<<<1024, 256, 0, s>>>(psd, n_det, row, k_lo, k_hi, df);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// <h_c|h_c>^i = 4 df sum_{k in band} f_k^{-7/3} / S^i[k] (Sec. II.D), fixed-order two-level reduction
// ------------------------------------------------------------------------------------------
constexpr int kSigmaBlocks = 256;

// stage 1: block b of detector i sums the band bins k = k_lo + b, k_lo + b + kSigmaBlocks, ... in a
// fixed tree order; stage 2 adds the kSigmaBlocks partials of each detector in order.
__global__ void sigma2_partial_kernel(const double* __restrict__ psd, int64_t row, int64_t k_lo, int64_t k_hi,
                                      double df, double* __restrict__ partial) {
    __shared__ double acc[256];
    const int i = blockIdx.y;
    double a = 0.0;
    for (int64_t k = k_lo + blockIdx.x + (int64_t)kSigmaBlocks * threadIdx.x; k <= k_hi;
         k += (int64_t)kSigmaBlocks * blockDim.x) {
        const double f = (double)k * df;
        a += pow(f, -7.0 / 3.0) / psd[i * row + k];
    }
    acc[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) acc[threadIdx.x] += acc[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[i * kSigmaBlocks + blockIdx.x] = acc[0];
}

__global__ void sigma2_final_kernel(const double* __restrict__ partial, double df, double* __restrict__ sigma2) {
    const int i = blockIdx.x;
    if (threadIdx.x != 0) return;
    double a = 0.0;
    for (int b = 0; b < kSigmaBlocks; ++b) a += partial[i * kSigmaBlocks + b];
    sigma2[i] = 4.0 * df * a;
}

// <h_c|h_c>^i = 4 df sum_{k in band} f_k^{-7/3} / S^i[k] (Sec. II.D); `work` holds n_det * 256 doubles
cudaError_t launch_sigma2(const double* psd, int n_det, int64_t row, int64_t k_lo, int64_t k_hi, double df,
                          double* sigma2, double* work, cudaStream_t s) {
    sigma2_partial_kernel<<<dim3(kSigmaBlocks, n_det), 256, 0, s>>>(psd, row, k_lo, k_hi, df, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sigma2_final_kernel<<<n_det, 32, 0, s>>>(work, df, sigma2);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// forward FFT of the zero-padded real data, binary64, same N = N1 N2 split as the fitness path:
// n = n1 + N1 n2, k = ka + N2 kb. Pass 1 transforms columns n1 over n2 and applies
// e^{-2 pi i n1 ka / N}; pass 2 transforms rows ka over n1 into natural order.
// ------------------------------------------------------------------------------------------
__host__ __device__ constexpr int create_v(int log_l) { return log_l >= 13 ? 8 : 4; }

template <int LOG_L>
__global__ void __launch_bounds__((1 << LOG_L) / create_v(LOG_L))
data_fft_pass1(const double* __restrict__ data, int64_t n_samples, int log_n1, const double2* __restrict__ tw,
               int tw_shift, const double2* __restrict__ twlo, const double2* __restrict__ twhi,
               double2* __restrict__ work) {
    constexpr int L = 1 << LOG_L;
    constexpr int kCreateV = create_v(LOG_L);
    constexpr int G = L / kCreateV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* smem = reinterpret_cast<double2*>(smem_raw);
    const int j = threadIdx.x;
    const int64_t n1 = blockIdx.x;
    const int i = blockIdx.y;
    const int64_t nn1 = (int64_t)1 << log_n1;
    const double* x = data + (int64_t)i * n_samples;
    double2 v[kCreateV];
#pragma unroll
    for (int q = 0; q < kCreateV; ++q) {
        const int64_t idx = n1 + nn1 * (j + q * G);
        v[q] = make_double2(idx < n_samples ? x[idx] : 0.0, 0.0);
    }
    block_fft<double, -1, LOG_L, kCreateV>(v, smem, 1, j, tw, tw_shift);
    double2* orow = work + (int64_t)i * L * nn1 + n1;
#pragma unroll
    for (int q = 0; q < kCreateV; ++q) {
        const int ta = j + q * G;
        const int m = (int)n1 * ta;
        const double2 w = cconj(cmul(twhi[m >> kTwLoBits], twlo[m & ((1 << kTwLoBits) - 1)]));
        orow[(int64_t)ta * nn1] = cmul(v[q], w);
    }
}

template <int LOG_L>
__global__ void __launch_bounds__((1 << LOG_L) / create_v(LOG_L))
data_fft_pass2(const double2* __restrict__ work, int log_n2, const double2* __restrict__ tw, int tw_shift,
               double2* __restrict__ spec) {
    constexpr int L = 1 << LOG_L;
    constexpr int kCreateV = create_v(LOG_L);
    constexpr int G = L / kCreateV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* smem = reinterpret_cast<double2*>(smem_raw);
    const int j = threadIdx.x;
    const int64_t ka = blockIdx.x;
    const int i = blockIdx.y;
    const int64_t n2 = (int64_t)1 << log_n2;
    const double2* row = work + ((int64_t)i * n2 + ka) * L;
    double2 v[kCreateV];
#pragma unroll
    for (int q = 0; q < kCreateV; ++q) v[q] = row[j + q * G];
    block_fft<double, -1, LOG_L, kCreateV>(v, smem, 1, j, tw, tw_shift);
    double2* out = spec + (int64_t)i * n2 * L;
#pragma unroll
    for (int q = 0; q < kCreateV; ++q) out[ka + n2 * (j + q * G)] = v[q];
}

template <int LG>
static cudaError_t data_fft_at(const double* data, int n_det, int64_t n_samples, int log_n1, int log_n2,
                               const double2* tw, int tw_shift_a, const double2* twlo, const double2* twhi,
                               double2* work, cudaStream_t s) {
    // pass 1 over columns of length N2 = 2^LG
    const size_t smem = sizeof(double2) << LG;
    auto k = data_fft_pass1<LG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)(1 << log_n1), (unsigned)n_det), (1 << LG) / create_v(LG), smem, s>>>(
        data, n_samples, log_n1, tw, tw_shift_a, twlo, twhi, work);
    (void)log_n2;
    return cudaGetLastError();
}

template <int LG>
static cudaError_t data_fft2_at(int n_det, int log_n2, const double2* tw, int tw_shift_b, const double2* work,
                                double2* spec, cudaStream_t s) {
    const size_t smem = sizeof(double2) << LG;
    auto k = data_fft_pass2<LG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)(1 << log_n2), (unsigned)n_det), (1 << LG) / create_v(LG), smem, s>>>(work, log_n2, tw, tw_shift_b,
                                                                                         spec);
    return cudaGetLastError();
}

cudaError_t launch_data_fft(const double* data, int n_det, int64_t n_samples, int log_n, int log_n1, int log_n2,
                            const double2* tw64, int tw_shift_a, int tw_shift_b, const double2* twlo64,
                            const double2* twhi64, double2* work, double2* spec, cudaStream_t s) {
    (void)log_n;
    cudaError_t e = cudaErrorInvalidValue;
    switch (log_n2) {
#define FCAS_CASE(LG) case LG: e = data_fft_at<LG>(data, n_det, n_samples, log_n1, log_n2, tw64, tw_shift_a, twlo64, twhi64, work, s); break;
        FCAS_CASE(2) FCAS_CASE(3) FCAS_CASE(4) FCAS_CASE(5) FCAS_CASE(6) FCAS_CASE(7) FCAS_CASE(8)
        FCAS_CASE(9) FCAS_CASE(10) FCAS_CASE(11) FCAS_CASE(12) FCAS_CASE(13)
#undef FCAS_CASE
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    switch (log_n1) {
#define FCAS_CASE(LG) case LG: return data_fft2_at<LG>(n_det, log_n2, tw64, tw_shift_b, work, spec, s);
        FCAS_CASE(2) FCAS_CASE(3) FCAS_CASE(4) FCAS_CASE(5) FCAS_CASE(6) FCAS_CASE(7) FCAS_CASE(8)
        FCAS_CASE(9) FCAS_CASE(10) FCAS_CASE(11) FCAS_CASE(12) FCAS_CASE(13)
#undef FCAS_CASE
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------------------------------
// Over-whitening (Sec. II.D) into the natural-order band spectrum kept by the context:
// ynat_i[k] = s 4 df f_k^{-7/6} e^{-i pi/4} dt X~_i[k] / S_i[k] for k in the band, 0 elsewhere
// (k < N/2; s the power-of-two scale).
// ------------------------------------------------------------------------------------------
__global__ void whiten_kernel(const double2* __restrict__ spec, const double* __restrict__ psd, int n_det,
                              int64_t psd_row, int log_n, int64_t k_lo, int64_t k_hi, double fs, double scale,
                              double2* __restrict__ ynat) {
    const int64_t n = (int64_t)1 << log_n;
    const int64_t half = n / 2;
    const double df = fs / (double)n;
    const double dt = 1.0 / fs;
    const double rs2 = 0.70710678118654752440;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < half * n_det;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(g / half);
        const int64_t k = g % half;
        double2 yv = make_double2(0.0, 0.0);
        if (k >= k_lo && k <= k_hi) {
            const double f = (double)k * df;
            const double2 x = spec[(int64_t)i * n + k];
            const double a = scale * 4.0 * df * pow(f, -7.0 / 6.0) * dt / psd[i * psd_row + k];
            // (x.re + i x.im) (1 - i) / sqrt 2
            yv = make_double2(a * rs2 * (x.x + x.y), a * rs2 * (x.y - x.x));
        }
        ynat[g] = yv;
    }
}

cudaError_t launch_whiten(const double2* spec, const double* psd, int n_det, int64_t psd_row, int log_n, int64_t k_lo,
                          int64_t k_hi, double fs, double scale, double2* ynat, cudaStream_t s) {
    whiten_kernel<<<4096, 256, 0, s>>>(spec, psd, n_det, psd_row, log_n, k_lo, k_hi, fs, scale, ynat);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Layout of the spectrum for pass A: Y as [k1 / K1B][i][k2 < N2/2][k1 % K1B] with k = k1 + N1 k2 (one
// detector's rows of a block adjacent; float pairs, binary64 pairs or float-float quadruples), and the chirp basis phi^-5/3, phi^-1, phi^-2/3, phi^-1/3
// (phi = f_k / f_*) in the order [k1 / K1B][k2][k1 % K1B] (float-float pairs in the FP32 form).
// ------------------------------------------------------------------------------------------
__global__ void layout_kernel(const double2* __restrict__ ynat, int n_det, int log_n, int log_n1, int log_n2, int k1b,
                              int64_t k_lo, int64_t k_hi, double fs, double f_star, int precision,
                              void* __restrict__ y, void* __restrict__ basis) {
    const int64_t n = (int64_t)1 << log_n;
    const int64_t half = n / 2;
    const int64_t n1 = (int64_t)1 << log_n1;
    const int64_t half2 = ((int64_t)1 << log_n2) / 2;
    const int64_t total = n1 * half2;
    const double df = fs / (double)n;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = g % k1b;
        const int64_t k2 = (g / k1b) % half2;
        const int64_t blk = g / (k1b * half2);
        const int64_t k = blk * k1b + c + n1 * k2;
        for (int i = 0; i < n_det; ++i) {
            const double2 yv = ynat[(int64_t)i * half + k];
            const int64_t yi = ((blk * n_det + i) * half2 + k2) * k1b + c;
            if (precision == FCAS_PREC_FP32) {
                static_cast<float2*>(y)[yi] = make_float2((float)yv.x, (float)yv.y);
            } else if (precision == FCAS_PREC_FF) {
                const float xh = (float)yv.x, ih = (float)yv.y;
                static_cast<float4*>(y)[yi] = make_float4(xh, (float)(yv.x - (double)xh), ih, (float)(yv.y - (double)ih));
            } else {
                static_cast<double2*>(y)[yi] = yv;
            }
        }
        double b53 = 0.0, b1 = 0.0, b23 = 0.0, b13 = 0.0;
        if (k >= k_lo && k <= k_hi) {
            b1 = f_star / ((double)k * df);
            b13 = cbrt(b1);
            b23 = b13 * b13;
            b53 = b1 * b23;
        }
        if (precision == FCAS_PREC_FP32) {
            // phi^-1/3 at every bin but DC, in the band and outside it (where the spectrum is zero): the
            // packed pass A forms the phase of the bins next to an anchor bin from the anchor's powers,
            // and the anchor of the band's lowest bins lies just below the band
            const double b13f = k >= k_lo && k <= k_hi ? b13 : k > 0 ? cbrt(f_star / ((double)k * df)) : 0.0;
            BasisF bf;
            bf.h = (float)b13f;
            bf.l = (float)(b13f - (double)bf.h);
            static_cast<BasisF*>(basis)[g] = bf;
        } else {
            BasisD bd;
            bd.a = make_double2(b53, b1);
            bd.b = make_double2(b23, b13);
            static_cast<BasisD*>(basis)[g] = bd;
        }
    }
}

cudaError_t launch_layout(const double2* ynat, int n_det, int log_n, int log_n1, int log_n2, int k1b, int64_t k_lo,
                          int64_t k_hi, double fs, double f_star, int precision, void* y, void* basis, cudaStream_t s) {
    if (k1b <= 0) return cudaErrorInvalidValue;
    layout_kernel<<<4096, 256, 0, s>>>(ynat, n_det, log_n, log_n1, log_n2, k1b, k_lo, k_hi, fs, f_star, precision, y,
                                       basis);
    return cudaGetLastError();
}

}  // namespace fcas
