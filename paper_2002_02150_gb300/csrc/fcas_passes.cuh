// Kernels of the two FFT passes of the fitness path and their launch dispatch, shared by the
// translation units that instantiate them for the FP32 / binary64 forms (fcas_kernels.cu) and the
// float-float form (fcas_kernels_ff.cu).
//
// Fitness path: per-particle geometry, pass A (fused template x data x delay phase feeding the
// first FFT pass), pass B (second FFT pass + antenna projection + partial argmax over t_c) and
// the final argmax. The length-N inverse transform over t_c is split as N = N1 N2 with
// k = k1 + N1 k2 and t = ta + N2 tb:
//   Z[ta + N2 tb] = sum_k1 e^{2 pi i k1 tb / N1} [ e^{2 pi i k1 ta / N} sum_k2 Q[k1 + N1 k2] e^{2 pi i k2 ta / N2} ]
// Pass A computes the bracket for every column k1 (length-N2 transforms) and stores it as
// A[ta][k1]; pass B transforms every row ta over k1 (length N1). Only two series per particle
// cross between the passes: the detector sum is taken with the network weights before the
// transform (see pass A).
#pragma once

#include <cfloat>
#include <climits>
#include <type_traits>

#include "fcas_fft16.cuh"
#include "fcas_kernels.cuh"

namespace fcas {

// ------------------------------------------------------------------------------------------
// Phase of Q_i[k] = Y_i[k] e^{2 pi i (psi(f_k)/2pi + f_k Delta^i)} (Sec. II.B, eq. data_template_innprod)
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ float round_nearest(float x) { return rintf(x); }
__device__ __forceinline__ double round_nearest(double x) { return rint(x); }

__device__ __forceinline__ double chirp_frac(const BasisD& b, const ParticleParams& pp) {
    double s = pp.c[0] * b.a.x + pp.c[1] * b.a.y + pp.c[2] * b.b.x + pp.c[3] * b.b.y;
    return s - rint(s);
}

// e^{2 pi i turns} for |turns| <= 1/2 with the hardware sine/cosine (absolute error ~4e-7 on
// [-pi, pi], far below the FP32 form's tolerance)
__device__ __forceinline__ float2 fast_phasor(float turns) {
    float sn, cs;
    __sincosf(6.2831853071795865f * turns, &sn, &cs);
    return make_float2(cs, sn);
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

// Entries of the float-float phasor table: e^{2 pi i m / kPhaseTab}, m < kPhaseTab.
constexpr int kPhaseTabBits = 10;
constexpr int kPhaseTab = 1 << kPhaseTabBits;

// e^{2 pi i u} in float-float for a float-float |u| <= 1/2 (or a binary64 u, split into two floats),
// on the FP32 units (table-driven reduction in the manner of Tang 1990): u = m / 1024 + r with the
// nearest table point m, and e^{2 pi i u} = T[m] (cos x + i sin x), x = 2 pi r, |x| <= pi / 1024. The
// remainder is exact in float-float (the table point subtracted exactly by a fused multiply-add);
// sin x = x - x^3/6 + x^5/120 and cos x = 1 - x^2/2 + x^4/24 (Taylor; the first omitted terms are
// below 2e-18), with x and x^2 in float-float and the small terms in float. Absolute error a few
// units of 2^-48.
__device__ __forceinline__ ff2 ff_unit_phasor(ffloat u, const ff2* __restrict__ tab) {
    const float uh = u.h, ul = u.l;
    const float m = rintf(uh * (float)kPhaseTab);
    float rl;
    const float rh = ff_two_sum(__fmaf_rn(m, -1.0f / (float)kPhaseTab, uh), ul, rl);
    const ffloat x = ff_mul(ffloat(rh, rl), ffloat(6.28318548202514648f, -1.74845553146951557e-7f));
    const ffloat x2 = ff_mul(x, x);
    // cos x = 1 - (x^2/2 - x^4/24)
    const ffloat hc = ff_add_f(ffloat(0.5f * x2.h, 0.5f * x2.l), -(x2.h * x2.h) * (1.0f / 24.0f));
    float e;
    const float ch = ff_fast_two_sum(1.0f, -hc.h, e);
    float cl;
    const float c = ff_fast_two_sum(ch, __fsub_rn(e, hc.l), cl);
    // sin x = x - x^3/6 (1 - x^2/20)
    const ffloat sn = ff_add_f(x, -(x.h * x2.h) * (1.0f / 6.0f) * __fmaf_rn(x2.h, -0.05f, 1.0f));
    const ff2 t = ldg_c(tab + ((int)m & (kPhaseTab - 1)));
    return cmul(t, ff2{ffloat(c, cl), sn});
}
__device__ __forceinline__ ff2 ff_unit_phasor(double u, const ff2* __restrict__ tab) {
    const float uh = __double2float_rn(u);
    return ff_unit_phasor(ffloat(uh, __double2float_rn(u - (double)uh)), tab);
}

// frac(k d) in float-float for an integer 0 <= k < 2^24 and d = d1 + d2 + d3 (three floats, each
// below half an ulp of the previous): k is exact in float, k d1 and k d2 are exact as products
// plus fused-multiply-add remainders, and k d3 is below 2^-24 |k d2|. Absolute error a few units of
// 2^-48 for |k d| < 2^8 turns, without binary64 arithmetic.
__device__ __forceinline__ ffloat ff_frac_mul_int(int k, float d1, float d2, float d3) {
    const float kf = (float)k;
    float p1 = __fmul_rn(kf, d1);
    const float e1 = __fmaf_rn(kf, d1, -p1);
    p1 = __fsub_rn(p1, rintf(p1));
    const float p2 = __fmul_rn(kf, d2);
    const float e2 = __fmaf_rn(kf, d2, -p2);
    float l1, l2;
    const float h1 = ff_two_sum(p1, p2, l1);
    const float h2 = ff_two_sum(e1, e2, l2);
    return ff_add_f(ff_add(ffloat(h1, l1), ffloat(h2, l2)), __fmul_rn(kf, d3));
}

// ------------------------------------------------------------------------------------------
// Pass A: for every band bin of the CTA's columns, Q_i[k] = Y_i[k] e^{2 pi i (psi(f_k)/2pi + f_k Delta^i)}
// is generated on the load and combined over detectors into the two network-weighted spectra
// P_a[k] = sum_i w_a,i Q_i[k] (a = 1, 2); each is transformed over k2 (length N2) and twiddled by
// e^{2 pi i k1 ta / N}. By linearity of the transform over t_c, Z-projections
// W_a(t) = sum_i w_a,i Z_i(t) are the transforms of P_a (Sec. II.C projection applied before the
// t_c scan instead of after it).
// ------------------------------------------------------------------------------------------
// Pass A's exchange padding: one spare element per 8 for 16-byte elements in radix-8 stages (their
// first-stage writes would otherwise fall two to a bank group), per 16 otherwise.
template <typename Real, int MAXRB>
__host__ __device__ constexpr int pass_a_pad_shift() {
    return sizeof(cplx<Real>) == 16 && MAXRB == 3 ? 3 : 4;
}
template <typename Real, int LOG_L, int K1B, int MAXRB>
__host__ __device__ constexpr int pass_a_buf_elems() {
    return K1B * xbuf_elems<pass_a_pad_shift<Real, MAXRB>()>(LOG_L);
}

// Pass A keeps two FFT exchange buffers when both fit in 200 KB of shared memory.
template <typename Real, int LOG_L, int K1B, int MAXRB>
__host__ __device__ constexpr bool pass_a_pingpong() {
    return 2 * sizeof(cplx<Real>) * (size_t)pass_a_buf_elems<Real, LOG_L, K1B, MAXRB>() <= 200 * 1024;
}

// The float-float form reduces the chirp phase in binary64 (basis as in the binary64 form) and the
// delay phase from a three-float split of the delay, and forms the phasors, the detector sums and
// everything after them in float-float.
template <typename Real> struct phase_of { using type = Real; };
template <> struct phase_of<ffloat> { using type = double; };
template <typename Real> using phase_t = typename phase_of<Real>::type;

// streamed store (evict-first): the intermediate is read back only by pass B
__device__ __forceinline__ void st_stream(float2* p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(double2* p, double2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(ff2* p, ff2 v) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(v.x.h, v.x.l, v.y.h, v.y.l));
}

template <typename Real>
struct DetConst {
    phase_t<Real> dh[FCAS_MAX_DET], dl[FCAS_MAX_DET];
    Real w1[FCAS_MAX_DET], w2[FCAS_MAX_DET];
};

template <typename Real, int LOG_L, int K1B, int MAXRB>
__global__ void __launch_bounds__(K1B * ((1 << LOG_L) / fftr_v(LOG_L, MAXRB)), 1)
pass_a_kernel(const cplx<Real>* __restrict__ y, const Basis<phase_t<Real>>* __restrict__ basis,
              const ParticleParams* __restrict__ params, int64_t p0, int64_t np, int n_det, int log_n1, int sub_req,
              cplx<Real>* __restrict__ out, const cplx<Real>* __restrict__ stw,
              const cplx<Real>* __restrict__ tw_lo, const cplx<Real>* __restrict__ tw_hi,
              const cplx<Real>* __restrict__ ptab) {
    using C = cplx<Real>;
    using P = phase_t<Real>;      // the real type of the phase reduction (binary64 for the float-float form)
    constexpr bool kFF = std::is_same<Real, ffloat>::value;
    constexpr int L = 1 << LOG_L;
    constexpr int V = fftr_v(LOG_L, MAXRB);
    constexpr int G = L / V;
    constexpr int VH = V / 2;    // values with k2 < L/2; the rest of the column is zero (k >= N/2)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    __shared__ DetConst<Real> sc;
    __shared__ float dsplit[3][FCAS_MAX_DET];   // float-float form: Delta^i df as three floats

    const int c = threadIdx.x % K1B;
    const int j = threadIdx.x / K1B;
    // CTA order: SUB adjacent column blocks of one particle, then the particles of the chunk, then
    // the next group of column blocks. The SUB CTAs fill whole 128-byte lines of each output row
    // together (so L2 merges them before write-back) and the chunk's particles read the same
    // spectrum block close in time (so it is fetched from DRAM once).
    const int nblk = (1 << log_n1) / K1B;
    const int sub = sub_req < nblk ? sub_req : nblk;
    const int64_t lin = blockIdx.x;
    const int64_t rest = lin / sub;
    const int64_t p = rest % np;
    const int blk = (int)((rest / np) * sub + lin % sub);
    const int k1 = blk * K1B + c;
    const ParticleParams* pp = params + p0 + p;
    if (!pp->valid) return;   // not evaluated (invalid input, or a PSO particle outside its box)
    if (threadIdx.x < FCAS_MAX_DET) {
        const int i = threadIdx.x;
        if constexpr (sizeof(P) == 4) {
            sc.dh[i] = pp->dh[i];
            sc.dl[i] = pp->dl[i];
            sc.w1[i] = pp->w1f[i];
            sc.w2[i] = pp->w2f[i];
        } else {
            sc.dh[i] = pp->dturn[i];
            sc.dl[i] = 0.0;
            sc.w1[i] = Real(pp->w1[i]);
            sc.w2[i] = Real(pp->w2[i]);
            if constexpr (kFF) {
                const double d = pp->dturn[i];
                const float d1 = (float)d;
                const float d2 = (float)(d - (double)d1);
                dsplit[0][i] = d1;
                dsplit[1][i] = d2;
                dsplit[2][i] = (float)(d - (double)d1 - (double)d2);
            }
        }
    }
    __syncthreads();
    const int n1 = 1 << log_n1;

    // Thread (c, j) owns the bins k = k1 + N1 (j + q G), q < VH. The delay phasors e^{2 pi i k Delta^i / T}
    // of consecutive q differ by the constant factor e^{2 pi i N1 G Delta^i / T}: one accurate phasor
    // and one step per detector, then products. The chirp phasor multiplies the detector sums last:
    // P_a[k] = e^{i psi(f_k)} sum_i w_a,i Y_i[k] e^{2 pi i f_k Delta^i}.
    C r1[VH], r2[VH];
#pragma unroll
    for (int q = 0; q < VH; ++q) r1[q] = r2[q] = mkc(Real(0.0f), Real(0.0f));
    // the chirp basis of the thread's bins is requested first: its latency overlaps the detector sums
    const Basis<P>* bb = basis + ((int64_t)blk * (L / 2) + j) * K1B + c;
    Basis<P> bq[sizeof(P) == 4 ? VH : 1];
    if constexpr (sizeof(P) == 4) {
#pragma unroll
        for (int q = 0; q < VH; ++q)
            if (FCAS_CHECK(((int64_t)blk * (L / 2) + j) * K1B + c + (int64_t)q * G * K1B < ((int64_t)L / 2 << log_n1),
                           kCheckBasis))
                bq[q] = bb[(int64_t)q * G * K1B];
    }
    const int kbase = k1 + n1 * j;
    const int kstep = n1 * G;
    const int64_t col0 = (int64_t)blk * n_det;
    // The float-float form keeps its code small (its fully unrolled double-word arithmetic would not
    // fit the instruction cache): the chirp phasors are formed in a loop into shared memory (the
    // transforms' exchange buffers, not yet in use) and the detector loop is not unrolled.
    if constexpr (kFF) {
#pragma unroll 1
        for (int q = 0; q < VH; ++q) {
            Basis<P> b{};
            if (FCAS_CHECK(((int64_t)blk * (L / 2) + j) * K1B + c + (int64_t)q * G * K1B < ((int64_t)L / 2 << log_n1),
                           kCheckBasis))
                b = bb[(int64_t)q * G * K1B];
            if (FCAS_CHECK((q * (int)blockDim.x + (int)threadIdx.x < pass_a_buf_elems<Real, LOG_L, K1B, MAXRB>()),
                           kCheckExchangeWrite))
                smem[q * blockDim.x + threadIdx.x] = ff_unit_phasor(chirp_frac(b, *pp), ptab);
        }
    }
    constexpr int kDetUnroll = kFF ? 1 : FCAS_MAX_DET;
#pragma unroll kDetUnroll
    for (int i = 0; i < FCAS_MAX_DET; ++i) {
        if (i >= n_det) break;
        C dph, dstep;
        if constexpr (sizeof(P) == 4) {
            float fb = frac_mul_ff((float)kbase, 0.0f, sc.dh[i], sc.dl[i]);
            float fs = frac_mul_ff((float)kstep, 0.0f, sc.dh[i], sc.dl[i]);
            fb -= rintf(fb);
            fs -= rintf(fs);
            dph = fast_phasor(fb);
            dstep = fast_phasor(fs);
        } else {
            if constexpr (kFF) {
                // the delay fraction without binary64 arithmetic (60-min pass A 34.7 -> 32.0 ms)
                dph = ff_unit_phasor(ff_frac_mul_int(kbase, dsplit[0][i], dsplit[1][i], dsplit[2][i]), ptab);
                dstep = ff_unit_phasor(ff_frac_mul_int(kstep, dsplit[0][i], dsplit[1][i], dsplit[2][i]), ptab);
            } else {
                const double fb = (double)kbase * sc.dh[i], fs = (double)kstep * sc.dh[i];
                dph = unit_phasor(fb - rint(fb));
                dstep = unit_phasor(fs - rint(fs));
            }
        }
        const C* yd = y + ((col0 + i) * (L / 2) + j) * K1B + c;
        const Real w1 = sc.w1[i], w2 = sc.w2[i];
#pragma unroll
        for (int q = 0; q < VH; ++q) {
            C yv = mkc(Real(0.0f), Real(0.0f));
            if (FCAS_CHECK(((col0 + i) * (L / 2) + j) * K1B + c + (int64_t)q * G * K1B <
                               (int64_t)n_det * ((int64_t)L / 2 << log_n1), kCheckSpectrum)) {
                if constexpr (kFF) yv = ldg_c(yd + (int64_t)q * G * K1B);
                else yv = yd[(int64_t)q * G * K1B];
            }
            const C t = cmul(yv, dph);
            r1[q].x += w1 * t.x;
            r1[q].y += w1 * t.y;
            r2[q].x += w2 * t.x;
            r2[q].y += w2 * t.y;
            if (q + 1 < VH) dph = cmul(dph, dstep);
        }
    }
    {
        float cfh[4], cfl[4];
        if constexpr (sizeof(P) == 4) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                cfh[r] = pp->ch[r];
                cfl[r] = pp->cl[r];
            }
        }
#pragma unroll
        for (int q = 0; q < VH; ++q) {
            C cp;
            if constexpr (sizeof(P) == 4) {
                const ChirpPowers b = chirp_powers_lean(bq[q]);
                float s = frac_mul_ff(cfh[0], cfl[0], b.b53.x, b.b53.y);
                s += frac_mul_ff(cfh[1], cfl[1], b.b1.x, b.b1.y);
                s += frac_mul_ff(cfh[2], cfl[2], b.b23.x, b.b23.y);
                s += frac_mul_ff(cfh[3], cfl[3], b.b13.x, b.b13.y);
                cp = fast_phasor(s - rintf(s));
            } else if constexpr (kFF) {
                cp = smem[q * blockDim.x + threadIdx.x];
            } else {
                Basis<P> b{};
                if (FCAS_CHECK(((int64_t)blk * (L / 2) + j) * K1B + c + (int64_t)q * G * K1B <
                                   ((int64_t)L / 2 << log_n1), kCheckBasis))
                    b = bb[(int64_t)q * G * K1B];
                cp = unit_phasor(chirp_frac(b, *pp));
            }
            r1[q] = cmul(r1[q], cp);
            r2[q] = cmul(r2[q], cp);
        }
    }
    if constexpr (kFF) __syncthreads();   // every chirp phasor read before the exchange buffers are reused

#pragma unroll 1
    for (int a = 0; a < kSeries; ++a) {
        C v[V];
#pragma unroll
        for (int q = 0; q < VH; ++q) v[q] = a == 0 ? r1[q] : r2[q];
#pragma unroll
        for (int q = VH; q < V; ++q) v[q] = mkc(Real(0.0f), Real(0.0f));
        // two exchange buffers where shared memory allows (no barrier before each exchange write); the
        // exchange count is continued across the series so that a buffer is never rewritten before
        // all its reads of the previous exchange are done
        constexpr int NX = (LOG_L + MAXRB - 1) / MAXRB - 1;
        // FP32: stage twiddles mostly loaded (60-min pass A 4.11 -> 4.07 ms; pass B keeps the
        // products, which need fewer registers than its three CTAs per SM allow for the loads)
        fftr<Real, +1, LOG_L, MAXRB, pass_a_pingpong<Real, LOG_L, K1B, MAXRB>(), 0, true, sizeof(Real) == 4,
             pass_a_pad_shift<Real, MAXRB>()>(v, smem + c, K1B, j, stw, pass_a_buf_elems<Real, LOG_L, K1B, MAXRB>(),
                                              (a * NX) & 1);
        C* orow = out + ((p * kSeries + a) * L) * (int64_t)n1 + k1;
        // e^{2 pi i k1 ta / N} for ta = j + q G: the value at q = 0 times powers of the step e^{2 pi i k1 G / N}
        const int m0 = k1 * j, ms = k1 * G;   // < N
        C w = cmul(ldg_c(tw_hi + (m0 >> kTwLoBits)), ldg_c(tw_lo + (m0 & ((1 << kTwLoBits) - 1))));
        const C step = cmul(ldg_c(tw_hi + (ms >> kTwLoBits)), ldg_c(tw_lo + (ms & ((1 << kTwLoBits) - 1))));
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int ta = j + q * G;
            if (FCAS_CHECK((p * kSeries + a) * (int64_t)L * n1 + k1 + (int64_t)ta * n1 < np * kSeries * (int64_t)L * n1,
                           kCheckInterWrite))
                st_stream(orow + (int64_t)ta * n1, cmul(v[q], w));   // streamed: read back only by pass B
            if (q + 1 < V) w = cmul(w, step);
        }
    }
}

// Argmax over the NT threads of a CTA of their (value, t) candidates, the lowest t among equal
// values; thread 0 writes the CTA's partial (t = INT_MAX: no candidate, written as -DBL_MAX).
template <int NT, typename Real>
__device__ __forceinline__ void cta_argmax_store(Real best, int bt, Real* red_v, int* red_t, Partial* out) {
    if constexpr (NT >= 32) {
        // NT is a multiple of 32: every warp is full
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const Real ov = shfl_down_r(best, off);
            const int ot = __shfl_down_sync(0xffffffffu, bt, off);
            if (ov > best || (ov == best && ot < bt)) { best = ov; bt = ot; }
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { red_v[warp] = best; red_t[warp] = bt; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < NT / 32; ++w)
                if (red_v[w] > best || (red_v[w] == best && red_t[w] < bt)) { best = red_v[w]; bt = red_t[w]; }
        }
    } else {
        // fewer than 32 threads: no shuffles over lanes that do not exist
        red_v[threadIdx.x] = best;
        red_t[threadIdx.x] = bt;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < NT; ++w)
                if (red_v[w] > best || (red_v[w] == best && red_t[w] < bt)) { best = red_v[w]; bt = red_t[w]; }
        }
    }
    if (threadIdx.x == 0)
        *out = Partial{bt == INT_MAX ? -DBL_MAX : to_double(best), bt == INT_MAX ? INT64_MAX : (int64_t)bt};
}

// ------------------------------------------------------------------------------------------
// Pass B: transforms every row ta of both series over k1 (length N1), Gamma^2(t) = |W1(t)|^2 +
// |W2(t)|^2 for t = ta + N2 tb (Sec. II.C, the maximisation over A_k in closed form), and the
// argmax over the CTA's rows (lowest t on ties).
// ------------------------------------------------------------------------------------------
// Resident pass-B CTAs per SM the compiler is held to: three for the FP32 form's 2^11- and
// 2^12-point rows (76-77 registers, no spills), two for other CTAs of up to 256 threads.
__host__ __device__ constexpr int pass_b_min_blocks(int log_l, int real_bytes) {
    return pass_b_threads(log_l, real_bytes) > 256 ? 1 : (real_bytes == 4 && (log_l == 11 || log_l == 12)) ? 3 : 2;
}

template <typename Real, int LOG_L>
__global__ void __launch_bounds__(pass_b_threads(LOG_L, sizeof(Real)), pass_b_min_blocks(LOG_L, sizeof(Real)))
pass_b_kernel(const cplx<Real>* __restrict__ inter, const ParticleParams* __restrict__ params, int64_t p0,
              int log_n2, int64_t n_samples, const cplx<Real>* __restrict__ stw, Partial* __restrict__ partials) {
    using C = cplx<Real>;
    constexpr int L = 1 << LOG_L;
    constexpr int V = shape_v(LOG_L);
    constexpr int G = L / V;
    constexpr int TB = pass_b_tb(LOG_L, sizeof(Real));
    constexpr int NT = TB * G;
    constexpr int BUF = fft16_buf_elems(LOG_L);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    constexpr int NRED = NT >= 32 ? NT / 32 : NT;
    __shared__ Real red_v[NRED];
    __shared__ int red_t[NRED];

    const int j = threadIdx.x % G;
    const int c = threadIdx.x / G;
    const int n2 = 1 << log_n2;
    const int ta = blockIdx.x * TB + c;
    const int64_t p = blockIdx.y;
    if (!params[p0 + p].valid) return;   // the final reduce reports NaN for it
    if constexpr (sizeof(Real) != 4) {
        // binary64 and float-float: the second series' row is requested into L2 now, so that its
        // loads after the first transform do not wait on DRAM (one 128-byte line per prefetch;
        // float-float pass B 20.0 -> 17.8 ms per 64 particles of the 60-min workload, FP32 unchanged)
        constexpr int LINE = 128 / (int)sizeof(C);
        const C* row1 = inter + ((p * kSeries + 1) * n2 + ta) * (int64_t)L;
        for (int e = j * LINE; e < L; e += G * LINE)
            if (FCAS_CHECK(((p * kSeries + 1) * n2 + ta) * (int64_t)L + e < (int64_t)gridDim.y * kSeries * n2 * L,
                           kCheckInterRead))
                asm volatile("prefetch.global.L2 [%0];" ::"l"(row1 + e));
    }

    Real g[V];
#pragma unroll
    for (int q = 0; q < V; ++q) g[q] = (Real)0;
#pragma unroll 1
    for (int a = 0; a < kSeries; ++a) {
        const C* row = inter + ((p * kSeries + a) * n2 + ta) * (int64_t)L;
        C v[V];
#pragma unroll
        for (int q = 0; q < V; ++q)
            if (FCAS_CHECK(((p * kSeries + a) * n2 + ta) * (int64_t)L + j + q * G < (int64_t)gridDim.y * kSeries * n2 * L,
                           kCheckInterRead))
                v[q] = row[j + q * G];
        fft16<Real, +1, LOG_L>(v, smem + c * BUF, 1, j, stw);
#pragma unroll
        for (int q = 0; q < V; ++q) g[q] += v[q].x * v[q].x + v[q].y * v[q].y;
    }
    // t = ta + N2 (j + q G) grows with q, so a strict comparison keeps the lowest t among equal values
    Real best = (Real)-1;
    int bt = INT_MAX;
#pragma unroll
    for (int q = 0; q < V; ++q) {
        const int t = ta + n2 * (j + q * G);
        if (t < n_samples && g[q] > best) {
            best = g[q];
            bt = t;
        }
    }
    cta_argmax_store<NT>(best, bt, red_v, red_t, partials + p * gridDim.x + blockIdx.x);
}

// ------------------------------------------------------------------------------------------
// FP32 form: both network-weighted series in one packed transform (fcas_x2.cuh). Lane 0 of every
// packed value is P_1 / W_1, lane 1 is P_2 / W_2; the intermediate holds one 16-byte element
// (re_1, re_2, im_1, im_2) per point, row-major: A[p][ta][k1].
// ------------------------------------------------------------------------------------------
__host__ __device__ constexpr int x2_a_threads(int log_l, int k1b, int maxrb = 4) {
    return k1b * ((1 << log_l) / fftr_v(log_l, maxrb));
}
// exchange padding: one spare element per 8 in radix-8 stages (their first-stage writes of 16-byte
// elements would otherwise fall two to a bank group), per 16 in radix-16 stages
__host__ __device__ constexpr int x2_pad_shift(int maxrb) { return maxrb == 3 ? 3 : 4; }
__host__ __device__ constexpr int x2_buf_elems(int log_l, int k1b, int maxrb = 4) {
    return maxrb == 3 ? k1b * xbuf_elems<3>(log_l) : k1b * xbuf_elems<4>(log_l);
}
// two exchange buffers when both fit in 200 KB of shared memory
__host__ __device__ constexpr bool x2_a_pingpong(int log_l, int k1b, int maxrb = 4) {
    return 2 * sizeof(c32x2) * (size_t)x2_buf_elems(log_l, k1b, maxrb) <= 200 * 1024;
}
// resident CTAs the compiler is held to: 512 threads' worth per SM with radix-16 stages (16 values per
// thread), 1024 threads' worth with radix-8 stages (8 values per thread)
__host__ __device__ constexpr int x2_min_blocks(int threads, int maxrb = 4) {
    return imin_c(16, imax_c(1, (maxrb == 3 ? 1024 : 512) / threads));
}

// Pass A of the FP32 form as a persistent grid: one wave of resident CTAs, each taking work items
// (particle, column block) blockIdx.x, blockIdx.x + gridDim.x, ... in the order of the other forms
// (SUB adjacent column blocks of one particle, then the particles of the chunk, then the next group of
// column blocks), so that one item's stores drain while the next item loads (60-min pass A 4.27 ->
// 4.07 ms per 64 particles against one item per CTA). Shapes with two exchange buffers run one item
// per CTA (the exchange parity restarts with every item). Each item requests its chirp basis and its
// first detector's spectrum before its particle's constants arrive (3.98 -> 3.83 ms; requesting more
// detectors early costs more in registers than it saves).
template <int LOG_L, int K1B, int MAXRB = 4>
__global__ void __launch_bounds__(x2_a_threads(LOG_L, K1B, MAXRB),
                                  x2_min_blocks(x2_a_threads(LOG_L, K1B, MAXRB), MAXRB))
pass_a_x2_kernel(const float2* __restrict__ y, const BasisF* __restrict__ basis,
                 const ParticleParams* __restrict__ params, int64_t p0, int64_t np, int n_det, int log_n1, int sub_req,
                 c32x2* __restrict__ out, const float2* __restrict__ stw, const float2* __restrict__ tw_lo,
                 const float2* __restrict__ tw_hi, int64_t items) {
    constexpr int L = 1 << LOG_L;
    constexpr int V = fftr_v(LOG_L, MAXRB);
    constexpr int G = L / V;
    constexpr int VH = V / 2;    // values with k2 < L/2; the rest of the column is zero (k >= N/2)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c32x2* smem = reinterpret_cast<c32x2*>(smem_raw);
    // the chirp phase from anchor bins shared by the lanes of adjacent columns (K1B of 2, 4 or 8)
    constexpr bool kLane = K1B >= 2 && K1B <= 8 && VH % K1B == 0;
    constexpr int kAnch = kLane ? VH / K1B : VH;   // basis loads (anchor bins) per lane

    const int c = threadIdx.x % K1B;
    const int j = threadIdx.x / K1B;
    const int nblk = (1 << log_n1) / K1B;
    const int sub = sub_req < nblk ? sub_req : nblk;
    const int n1 = 1 << log_n1;
#pragma unroll 1
    for (int64_t lin = blockIdx.x; lin < items; lin += gridDim.x) {
        const int64_t rest = lin / sub;
        const int64_t p = rest % np;
        const int blk = (int)((rest / np) * sub + lin % sub);
        const int k1 = blk * K1B + c;
        const ParticleParams* pp = params + p0 + p;
        // the chirp basis and the first detector's spectrum of the thread's bins do not depend on the
        // particle: requested before its constants, so that the two round trips overlap
        BasisF bq[kAnch];
        if constexpr (kLane) {
            // the basis of the lane's anchor bins: the lane group's first column (K1B blk) at
            // q = c kAnch + a
            const int64_t bidx0 = ((int64_t)blk * (L / 2) + j) * K1B;
#pragma unroll
            for (int a = 0; a < kAnch; ++a) {
                const int64_t bi = bidx0 + (int64_t)(c * kAnch + a) * G * K1B;
                if (FCAS_CHECK(bi < ((int64_t)L / 2 << log_n1), kCheckBasis)) bq[a] = basis[bi];
            }
        } else {
            const int64_t bidx0 = ((int64_t)blk * (L / 2) + j) * K1B + c;
#pragma unroll
            for (int q = 0; q < VH; ++q)
                if (FCAS_CHECK(bidx0 + (int64_t)q * G * K1B < ((int64_t)L / 2 << log_n1), kCheckBasis))
                    bq[q] = basis[bidx0 + (int64_t)q * G * K1B];
        }
        const int64_t col0 = (int64_t)blk * n_det;
        float2 y0[VH];   // detector 0 (every context has at least one)
        {
            const int64_t yidx0 = (col0 * (L / 2) + j) * K1B + c;
#pragma unroll
            for (int q = 0; q < VH; ++q) {
                y0[q] = make_float2(0.0f, 0.0f);
                if (FCAS_CHECK(yidx0 + (int64_t)q * G * K1B < (int64_t)n_det * ((int64_t)L / 2 << log_n1),
                               kCheckSpectrum))
                    y0[q] = y[yidx0 + (int64_t)q * G * K1B];
            }
        }
        // The particle's constants are read where they are used, straight from its parameter record
        // (the same address across the CTA, cached in L1): no shared-memory copy and no barrier before
        // the detector sums (60-min pass A 3.75 -> 3.67 ms per 64 particles).
        const int taylor_ok = pp->taylor_ok;
        if (!pp->valid) continue;   // not evaluated (invalid input, or a PSO particle outside its box)

        // Thread (c, j) owns the bins k = k1 + N1 (j + q G), q < VH: the detector sums per series with
        // the delay phasors by recurrence, then the chirp phasor (as in the other forms), in scalar FP32.
        float2 r1[VH], r2[VH];
#pragma unroll
        for (int q = 0; q < VH; ++q) r1[q] = r2[q] = make_float2(0.0f, 0.0f);
        const int kbase = k1 + n1 * j;
#pragma unroll
        for (int i = 0; i < FCAS_MAX_DET; ++i) {
            if (i >= n_det) break;
            // the phasor at the thread's first bin; its step to the next bin (kstep further) is the
            // particle's (formed once by the geometry kernel for this shape)
            float fb = frac_mul_ff((float)kbase, 0.0f, __ldg(&pp->dh[i]), __ldg(&pp->dl[i]));
            fb -= rintf(fb);
            float2 dph = fast_phasor(fb);
            const float2 dstep = __ldg(&pp->dstep[i]);
            const int64_t yidx0 = ((col0 + i) * (L / 2) + j) * K1B + c;
            const float2* yd = y + yidx0;
            const float w1 = __ldg(&pp->w1f[i]), w2 = __ldg(&pp->w2f[i]);
#pragma unroll
            for (int q = 0; q < VH; ++q) {
                float2 yv = make_float2(0.0f, 0.0f);
                if (i == 0)
                    yv = y0[q];
                else if (FCAS_CHECK(yidx0 + (int64_t)q * G * K1B < (int64_t)n_det * ((int64_t)L / 2 << log_n1),
                               kCheckSpectrum))
                    yv = yd[(int64_t)q * G * K1B];
                const float2 t = cmul(yv, dph);
                r1[q].x += w1 * t.x;
                r1[q].y += w1 * t.y;
                r2[q].x += w2 * t.x;
                r2[q].y += w2 * t.y;
                if (q + 1 < VH) dph = cmul(dph, dstep);
            }
        }
        c32x2 v[V];
        {
            float cfh[4], cfl[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                cfh[r] = __ldg(&pp->ch[r]);
                cfl[r] = __ldg(&pp->cl[r]);
            }
            if (kLane && (taylor_ok & (K1B <= 4 ? 1 : 2))) {
                // The K1B lanes of a group (consecutive lanes, one per column) hold the adjacent bins
                // k_a + c (c < K1B) at every q. Lane c forms, at the anchor bins k_a of kAnch values of
                // q, the phase psi (turns: float-float products reduced mod 1) and in FP32 from the same
                // powers b_m = phi^-e_m (e_m = 5/3, 1, 2/3, 1/3) its derivatives along k:
                //   psi' = -(1/k) sum_m e_m c_m b_m,   psi'' = (1/k^2) sum_m e_m (e_m + 1) c_m b_m.
                // The group exchanges them and each lane steps to its own bin by
                //   psi(k_a + c) = psi(k_a) + c psi' + c^2 psi''/2;
                // taylor_ok (set by the geometry kernel: bit 0 for steps of up to 3 bins, bit 1 up to 7)
                // bounds the remainder below 1e-7 turns for the particle; otherwise every bin's phase
                // is formed from its own powers.
                float sa[kAnch], d1a[kAnch], d2a[kAnch];
#pragma unroll
                for (int a = 0; a < kAnch; ++a) {
                    const ChirpPowers b = chirp_powers_lean(bq[a]);
                    float s = frac_mul_ff(cfh[0], cfl[0], b.b53.x, b.b53.y);
                    s += frac_mul_ff(cfh[1], cfl[1], b.b1.x, b.b1.y);
                    s += frac_mul_ff(cfh[2], cfl[2], b.b23.x, b.b23.y);
                    s += frac_mul_ff(cfh[3], cfl[3], b.b13.x, b.b13.y);
                    const float g1 =
                        fmaf(cfh[0] * (5.0f / 3.0f), b.b53.x,
                             fmaf(cfh[1], b.b1.x, fmaf(cfh[2] * (2.0f / 3.0f), b.b23.x, cfh[3] * (1.0f / 3.0f) * b.b13.x)));
                    const float g2 =
                        fmaf(cfh[0] * (40.0f / 9.0f), b.b53.x,
                             fmaf(cfh[1] * 2.0f, b.b1.x, fmaf(cfh[2] * (10.0f / 9.0f), b.b23.x, cfh[3] * (4.0f / 9.0f) * b.b13.x)));
                    const float ka = (float)(blk * K1B + n1 * (j + (c * kAnch + a) * G));   // < 2^24: exact
                    const float rk = ka > 0.0f ? __frcp_rn(ka) : 0.0f;   // the DC bin carries no phase
                    sa[a] = s;
                    d1a[a] = -g1 * rk;
                    d2a[a] = 0.5f * g2 * rk * rk;
                }
                const int lane0 = (threadIdx.x & 31) - c;   // the group's first lane
                const float cf = (float)c;
#pragma unroll
                for (int q = 0; q < VH; ++q) {
                    const int src = lane0 + q / kAnch;
                    const float s0 = __shfl_sync(0xffffffffu, sa[q % kAnch], src);
                    const float d1 = __shfl_sync(0xffffffffu, d1a[q % kAnch], src);
                    const float d2 = __shfl_sync(0xffffffffu, d2a[q % kAnch], src);
                    const float s = fmaf(cf, fmaf(cf, d2, d1), s0);
                    const float2 cp = fast_phasor(s - rintf(s));
                    v[q] = pack_series(cmul(r1[q], cp), cmul(r2[q], cp));
                }
            } else {
                // every bin from its own basis entry (requested here when only the anchors' were)
                BasisF bo[VH];
                if constexpr (kLane) {
                    const int64_t bidx0 = ((int64_t)blk * (L / 2) + j) * K1B + c;
#pragma unroll
                    for (int q = 0; q < VH; ++q)
                        if (FCAS_CHECK(bidx0 + (int64_t)q * G * K1B < ((int64_t)L / 2 << log_n1), kCheckBasis))
                            bo[q] = basis[bidx0 + (int64_t)q * G * K1B];
                } else {
#pragma unroll
                    for (int q = 0; q < VH; ++q) bo[q] = bq[q < kAnch ? q : 0];
                }
#pragma unroll
                for (int q = 0; q < VH; ++q) {
                    const ChirpPowers b = chirp_powers_lean(bo[q]);
                    float s = frac_mul_ff(cfh[0], cfl[0], b.b53.x, b.b53.y);
                    s += frac_mul_ff(cfh[1], cfl[1], b.b1.x, b.b1.y);
                    s += frac_mul_ff(cfh[2], cfl[2], b.b23.x, b.b23.y);
                    s += frac_mul_ff(cfh[3], cfl[3], b.b13.x, b.b13.y);
                    const float2 cp = fast_phasor(s - rintf(s));
                    v[q] = pack_series(cmul(r1[q], cp), cmul(r2[q], cp));
                }
            }
        }
#pragma unroll
        for (int q = VH; q < V; ++q) v[q] = zero_c32x2();
        // one transform of both series; stage twiddles w^r (r < 4) and w^{4h} loaded, the rest one
        // product each (formed once for both series)
        fftr<x2f, +1, LOG_L, MAXRB, x2_a_pingpong(LOG_L, K1B, MAXRB), 0, true, true, x2_pad_shift(MAXRB)>(
            v, smem + c, K1B, j, stw, x2_buf_elems(LOG_L, K1B, MAXRB), 0);
        c32x2* orow = out + ((int64_t)p * L) * n1 + k1;
        // e^{2 pi i k1 ta / N} for ta = j + q G: the value at q = 0 times powers of the step e^{2 pi i k1 G / N}
        const int m0 = k1 * j, ms = k1 * G;   // < N
        float2 w = cmul(__ldg(tw_hi + (m0 >> kTwLoBits)), __ldg(tw_lo + (m0 & ((1 << kTwLoBits) - 1))));
        const float2 step = cmul(__ldg(tw_hi + (ms >> kTwLoBits)), __ldg(tw_lo + (ms & ((1 << kTwLoBits) - 1))));
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int ta = j + q * G;
            if (FCAS_CHECK((int64_t)p * L * n1 + k1 + (int64_t)ta * n1 < np * (int64_t)L * n1, kCheckInterWrite))
                st_stream_x2(orow + (int64_t)ta * n1, cmul(v[q], w));   // streamed: read back only by pass B
            if (q + 1 < V) w = cmul(w, step);
        }
    }
}

__host__ __device__ constexpr int x2_b_threads(int log_l) { return pass_b_threads(log_l, 4); }
// resident pass-B CTAs the compiler is held to: two of 256 threads (16 values per thread)
__host__ __device__ constexpr int x2_b_min_blocks(int log_l) { return x2_b_threads(log_l) > 256 ? 1 : 2; }

template <int LOG_L>
__global__ void __launch_bounds__(x2_b_threads(LOG_L), x2_b_min_blocks(LOG_L))
pass_b_x2_kernel(const c32x2* __restrict__ inter, const ParticleParams* __restrict__ params, int64_t p0, int log_n2,
                 int64_t n_samples, const float2* __restrict__ stw, Partial* __restrict__ partials, int64_t ahead) {
    constexpr int L = 1 << LOG_L;
    constexpr int V = shape_v(LOG_L);
    constexpr int G = L / V;
    constexpr int TB = pass_b_tb(LOG_L, 4);
    constexpr int NT = TB * G;
    constexpr int BUF = fft16_buf_elems(LOG_L);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c32x2* smem = reinterpret_cast<c32x2*>(smem_raw);
    constexpr int NRED = NT >= 32 ? NT / 32 : NT;
    __shared__ float red_v[NRED];
    __shared__ int red_t[NRED];

    const int j = threadIdx.x % G;
    const int c = threadIdx.x / G;
    const int n2 = 1 << log_n2;
    const int ta = blockIdx.x * TB + c;
    const int64_t p = blockIdx.y;
    // The rows of the CTA `ahead` places later in launch order (one wave of resident CTAs) are requested
    // into L2 by one bulk prefetch per warp, so that DRAM keeps streaming while the resident CTAs
    // transform (60-min pass B 2.10 -> 1.94 ms per 64 particles).
    if constexpr (NT >= 32 && NT % 32 == 0) {
        if ((threadIdx.x & 31) == 0 && ahead > 0) {
            const int64_t nxt = (int64_t)blockIdx.y * gridDim.x + blockIdx.x + ahead;
            constexpr unsigned kBytes = (unsigned)(TB * L * sizeof(c32x2) / (NT / 32));   // 512 V bytes
            const int64_t e0 = ((nxt / gridDim.x) * n2 + (nxt % gridDim.x) * TB) * L +
                               (threadIdx.x >> 5) * (kBytes / sizeof(c32x2));
            if (nxt < (int64_t)gridDim.x * gridDim.y &&
                FCAS_CHECK(e0 + kBytes / sizeof(c32x2) <= (int64_t)gridDim.y * n2 * L, kCheckInterRead)) {
                const c32x2* src = inter + e0;
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(src)),
                             "r"(kBytes)
                             : "memory");
            }
        }
    }
    if (!params[p0 + p].valid) return;   // the final reduce reports NaN for it
    const int64_t row0 = ((int64_t)p * n2 + ta) * L;
    const c32x2* row = inter + row0;
    c32x2 v[V];
#pragma unroll
    for (int q = 0; q < V; ++q) {
        v[q] = zero_c32x2();
        if (FCAS_CHECK(row0 + j + q * G < (int64_t)gridDim.y * n2 * L, kCheckInterRead))
            v[q] = ld_na(row + j + q * G);   // read once: no L1 allocation (60-min pass B 2.13 -> 2.10 ms)
    }
    fft16<x2f, +1, LOG_L>(v, smem + c * BUF, 1, j, stw);
    // Gamma^2(t) = |W_1(t)|^2 + |W_2(t)|^2; t = ta + N2 (j + q G) grows with q, so a strict
    // comparison keeps the lowest t among equal values
    float best = -1.0f;
    int bt = INT_MAX;
    // the lag bound in 32 bits (t < N <= 2^24): one comparison per value instead of a 64-bit one
    // (60-min pass B 1.95 -> 1.87 ms per 64 particles)
    const int ns = n_samples < (int64_t)INT_MAX ? (int)n_samples : INT_MAX;
#pragma unroll
    for (int q = 0; q < V; ++q) {
        const int t = ta + n2 * (j + q * G);
        const float g = norm2_sum(v[q]);
        if (t < ns && g > best) {
            best = g;
            bt = t;
        }
    }
    cta_argmax_store<NT>(best, bt, red_v, red_t, partials + p * gridDim.x + blockIdx.x);
}

// Column-block widths of the packed FP32 pass A: the default of the length and, from 2^8 points on,
// half and twice it while a CTA stays within 512 threads.
template <int LG>
constexpr bool x2_k1b_ok(int k) {
    return k >= 1 && k <= 16 && k <= (1 << LG) && x2_a_threads(LG, k) <= 512;
}

template <int LG, int K1B, int MAXRB = 4>
static cudaError_t pass_a_x2_at(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np,
                                void* inter, cudaStream_t s) {
    constexpr int THREADS = x2_a_threads(LG, K1B, MAXRB);
    const size_t smem =
        (x2_a_pingpong(LG, K1B, MAXRB) ? 2 : 1) * sizeof(c32x2) * (size_t)x2_buf_elems(LG, K1B, MAXRB);
    auto kern = pass_a_x2_kernel<LG, K1B, MAXRB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t items = np * ((1 << pl.log_n1) / K1B);
    int64_t ctas = items;
    if constexpr (!x2_a_pingpong(LG, K1B, MAXRB)) {
        // one wave: the resident CTAs of every SM
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
        if (e != cudaSuccess) return e;
        const int64_t wave = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
        if (wave < ctas) ctas = wave;
    }
    kern<<<(unsigned)ctas, THREADS, smem, s>>>(static_cast<const float2*>(pl.y), static_cast<const BasisF*>(pl.basis),
                                               params, p0, np, pl.n_det, pl.log_n1, pl.sub, static_cast<c32x2*>(inter),
                                               static_cast<const float2*>(pl.stw_a), static_cast<const float2*>(pl.tw_lo),
                                               static_cast<const float2*>(pl.tw_hi), items);
    return cudaGetLastError();
}

template <int LG>
static cudaError_t pass_a_x2_lg(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np,
                                void* inter, cudaStream_t s) {
    constexpr int KD = pass_a_k1b(LG, 4);
    if (pl.radix_bits_a == 3) {
        // radix-8 stages: 8 values per thread, CTAs of 2 or 4 columns (at most 1024 threads)
        if constexpr (LG >= 10 && LG <= 11)
            if (pl.k1b == 4) return pass_a_x2_at<LG, 4, 3>(pl, params, p0, np, inter, s);
        if constexpr (LG >= 10 && LG <= 12)
            if (pl.k1b == 2) return pass_a_x2_at<LG, 2, 3>(pl, params, p0, np, inter, s);
        return cudaErrorInvalidValue;
    }
    if (pl.radix_bits_a != 4) return cudaErrorInvalidValue;
    if (pl.k1b == KD) return pass_a_x2_at<LG, KD>(pl, params, p0, np, inter, s);
    if constexpr (LG >= 10 && KD > 1)
        if (pl.k1b == 1) return pass_a_x2_at<LG, 1>(pl, params, p0, np, inter, s);   // one column per CTA
    if constexpr (LG >= 8) {
        if constexpr (x2_k1b_ok<LG>(KD / 2))
            if (pl.k1b == KD / 2) return pass_a_x2_at<LG, (KD / 2 > 0 ? KD / 2 : 1)>(pl, params, p0, np, inter, s);
        if constexpr (x2_k1b_ok<LG>(KD * 2))
            if (pl.k1b == KD * 2) return pass_a_x2_at<LG, (KD * 2 <= 16 ? KD * 2 : 16)>(pl, params, p0, np, inter, s);
    }
    return cudaErrorInvalidValue;
}

template <int LG>
static cudaError_t pass_b_x2_at(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np,
                                const void* inter, Partial* partials, cudaStream_t s) {
    constexpr int TB = pass_b_tb(LG, 4);
    const size_t smem = sizeof(c32x2) * (size_t)TB * fft16_buf_elems(LG);
    auto kern = pass_b_x2_kernel<LG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, x2_b_threads(LG), smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((1 << pl.log_n2) / TB), (unsigned)np);
    kern<<<grid, x2_b_threads(LG), smem, s>>>(static_cast<const c32x2*>(inter), params, p0, pl.log_n2, pl.n_samples,
                                              static_cast<const float2*>(pl.stw_b), partials,
                                              (int64_t)sms * (per_sm > 0 ? per_sm : 1));
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// dispatch on the transform lengths
// ------------------------------------------------------------------------------------------
#define FCAS_LOG_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13)

template <typename Real, int LG, int K1B, int MAXRB = 4>
static cudaError_t pass_a_at(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np, void* inter,
                             cudaStream_t s) {
    constexpr int THREADS = K1B * ((1 << LG) / fftr_v(LG, MAXRB));
    const size_t smem = (pass_a_pingpong<Real, LG, K1B, MAXRB>() ? 2 : 1) * sizeof(cplx<Real>) *
                        (size_t)pass_a_buf_elems<Real, LG, K1B, MAXRB>();
    auto kern = pass_a_kernel<Real, LG, K1B, MAXRB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ctas = np * ((1 << pl.log_n1) / K1B);
    kern<<<(unsigned)ctas, THREADS, smem, s>>>(static_cast<const cplx<Real>*>(pl.y),
                                     static_cast<const Basis<phase_t<Real>>*>(pl.basis),
                                     params, p0, np, pl.n_det, pl.log_n1, pl.sub, static_cast<cplx<Real>*>(inter),
                                     static_cast<const cplx<Real>*>(pl.stw_a), static_cast<const cplx<Real>*>(pl.tw_lo),
                                     static_cast<const cplx<Real>*>(pl.tw_hi), static_cast<const cplx<Real>*>(pl.ptab));
    return cudaGetLastError();
}

// Column-block widths compiled for pass A: the default of the length and, for the FP32 form at
// lengths >= 2^8, half and twice it (the autotuner's choices).
template <int LG, int RB>
constexpr bool k1b_variant_ok(int k) {
    return k >= 1 && k <= 16 && k <= (1 << LG) && k * ((1 << LG) / shape_v(LG)) <= 1024;
}

template <typename Real, int LG>
static cudaError_t pass_a_lg(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np,
                             void* inter, cudaStream_t s) {
    constexpr int RB = sizeof(Real);
    constexpr int KD = pass_a_k1b(LG, RB);
    if (pl.radix_bits_a == 3) {
        // radix-8 stages: 8 values per thread, 1024-thread CTAs of 4 columns (FP32, >= 2^10 points)
        if constexpr (RB == 4 && LG >= 10 && LG <= 12)
            if (pl.k1b == 4) return pass_a_at<Real, LG, 4, 3>(pl, params, p0, np, inter, s);
        // float-float: 512-thread CTAs of 2 columns (half the registers per thread of radix 16)
        if constexpr (std::is_same<Real, ffloat>::value && LG >= 10 && LG <= 12)
            if (pl.k1b == 2) return pass_a_at<Real, LG, 2, 3>(pl, params, p0, np, inter, s);
        return cudaErrorInvalidValue;
    }
    if (pl.k1b == KD) return pass_a_at<Real, LG, KD>(pl, params, p0, np, inter, s);
    if constexpr (RB == 4 && LG >= 8) {
        if constexpr (k1b_variant_ok<LG, RB>(KD / 2))
            if (pl.k1b == KD / 2) return pass_a_at<Real, LG, (KD / 2 > 0 ? KD / 2 : 1)>(pl, params, p0, np, inter, s);
        if constexpr (k1b_variant_ok<LG, RB>(KD * 2))
            if (pl.k1b == KD * 2) return pass_a_at<Real, LG, (KD * 2 <= 16 ? KD * 2 : 16)>(pl, params, p0, np, inter, s);
    }
    return cudaErrorInvalidValue;
}

template <typename Real, int LG>
static cudaError_t pass_b_at(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np,
                             const void* inter, Partial* partials, cudaStream_t s) {
    constexpr int TB = pass_b_tb(LG, sizeof(Real));
    constexpr int THREADS = pass_b_threads(LG, sizeof(Real));
    const size_t smem = sizeof(cplx<Real>) * (size_t)TB * fft16_buf_elems(LG);
    auto kern = pass_b_kernel<Real, LG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((1 << pl.log_n2) / TB), (unsigned)np);
    kern<<<grid, THREADS, smem, s>>>(static_cast<const cplx<Real>*>(inter), params, p0, pl.log_n2, pl.n_samples,
                                     static_cast<const cplx<Real>*>(pl.stw_b), partials);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_pass_a(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np, void* inter,
                          cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if constexpr (std::is_same<Real, float>::value) {
        // the FP32 form: both series in one packed transform
        switch (pl.log_n2) {
#define FCAS_CASE(LG) case LG: return pass_a_x2_lg<LG>(pl, params, p0, np, inter, s);
            FCAS_LOG_CASES(FCAS_CASE)
#undef FCAS_CASE
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (pl.log_n2) {
#define FCAS_CASE(LG) case LG: return pass_a_lg<Real, LG>(pl, params, p0, np, inter, s);
            FCAS_LOG_CASES(FCAS_CASE)
#undef FCAS_CASE
            default: return cudaErrorInvalidValue;
        }
    }
}

template <typename Real>
cudaError_t launch_pass_b(const FitnessPlan& pl, const ParticleParams* params, int64_t p0, int64_t np,
                          const void* inter, Partial* partials, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if constexpr (std::is_same<Real, float>::value) {
        switch (pl.log_n1) {
#define FCAS_CASE(LG) case LG: return pass_b_x2_at<LG>(pl, params, p0, np, inter, partials, s);
            FCAS_LOG_CASES(FCAS_CASE)
#undef FCAS_CASE
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (pl.log_n1) {
#define FCAS_CASE(LG) case LG: return pass_b_at<Real, LG>(pl, params, p0, np, inter, partials, s);
            FCAS_LOG_CASES(FCAS_CASE)
#undef FCAS_CASE
            default: return cudaErrorInvalidValue;
        }
    }
}

}  // namespace fcas
