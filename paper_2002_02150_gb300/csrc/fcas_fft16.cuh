// Register-resident Stockham FFT with radix-16 stages, used by both passes of the fitness path.
//
// A transform of length L = 2^LOG_L (L >= 16) is held by G = L / 16 threads, thread j owning the
// 16 values at positions j + q G (q = 0..15) on entry and on exit (natural order). Stage s has
// radix R_s = 16 while at least four bits of L remain, then one stage takes the remaining 1-3
// bits; for L < 16 a single stage of radix L is used (V = L values per thread, G = 1). The same
// code with radix-8 full stages (8 values per thread, twice the threads) trades one more
// shared-memory exchange for half the registers. Each stage
// is the Stockham self-sorting step: task jj reads x[jj + r L/R], multiplies by
// e^{S 2 pi i r (jj mod Ns) / (Ns R)}, applies the R-point DFT in registers and writes to
// (jj / Ns) Ns R + (jj mod Ns) + r Ns. Consecutive stages exchange data through shared memory,
// padded by one element every 16 so that the stride-16 writes of a stage do not share banks.
// With PP the exchanges alternate between two buffers `alt` elements apart (exchange e of the
// transform uses buffer (e + par0) mod 2): a buffer is rewritten only two exchanges after it was
// last read, with a barrier in between, so the barrier before each write is dropped.
// Twiddles come from a per-length table laid out stage by stage as
//   T[(Ns - 1) + (r - 1) Ns + jm] = e^{2 pi i r jm / (Ns R)},   r = 1..R-1, jm = 0..Ns-1,
// so that a warp reads consecutive entries; the stages together use L - 1 entries.
#pragma once

#include <type_traits>

#include "fcas_internal.cuh"
#include "fcas_ff.cuh"
#include "fcas_x2.cuh"

namespace fcas {

template <> struct cplx_of<ffloat> { using type = ff2; };

// Element type of the per-stage twiddle tables of a transform over cplx<Real> values: the value type
// itself, except for the packed two-series form, whose lanes share one scalar twiddle.
template <typename Real> struct fft_tw_of { using type = cplx<Real>; };
template <> struct fft_tw_of<x2f> { using type = float2; };
template <typename Real> using fft_tw = typename fft_tw_of<Real>::type;
__device__ __forceinline__ float2 tw_one(float2) { return make_float2(1.0f, 0.0f); }
__device__ __forceinline__ double2 tw_one(double2) { return make_double2(1.0, 0.0); }
__device__ __forceinline__ ff2 tw_one(ff2) { return ff2{ffloat(1.0f, 0.0f), ffloat(0.0f, 0.0f)}; }

// a + S i b and a - S i b (S = +1 or -1), the multiplication by +-i folded into the addition
template <int S, typename C> __device__ __forceinline__ C add_si(C a, C b) {
    return S > 0 ? mkc(a.x - b.y, a.y + b.x) : mkc(a.x + b.y, a.y - b.x);
}
template <int S, typename C> __device__ __forceinline__ C sub_si(C a, C b) { return add_si<-S>(a, b); }

// read-only cached load of a complex table entry
__device__ __forceinline__ float2 ldg_c(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_c(const double2* p) { return __ldg(p); }
__device__ __forceinline__ ff2 ldg_c(const ff2* p) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    return ff2{ffloat(q.x, q.y), ffloat(q.z, q.w)};
}
template <int SGN, typename R> __device__ __forceinline__ R sgn_mul(R v) { return SGN > 0 ? v : -v; }

// MAXRB: radix bits of the full stages (4: radix 16, 16 values per thread; 3: radix 8, 8 values)
__host__ __device__ constexpr int fftr_radix_bits(int log_l, int done, int maxrb) {
    return (log_l - done) >= maxrb ? maxrb : (log_l - done);
}
__host__ __device__ constexpr int fftr_v(int log_l, int maxrb) { return log_l >= maxrb ? (1 << maxrb) : (1 << log_l); }
__host__ __device__ constexpr int fft16_radix_bits(int log_l, int done) { return fftr_radix_bits(log_l, done, 4); }
__host__ __device__ constexpr int fft16_v(int log_l) { return fftr_v(log_l, 4); }
__host__ __device__ constexpr int fft16_pad(int e) { return e + (e >> 4); }
__host__ __device__ constexpr int fft16_buf_elems(int log_l) { return fft16_pad(1 << log_l); }
// the exchange padding with one spare element per 2^PS (PS = 4 above; 3 for 16-byte elements in
// radix-8 stages, whose first-stage writes would otherwise fall two to a bank group)
template <int PS> __host__ __device__ constexpr int xpad(int e) { return e + (e >> PS); }
template <int PS> __host__ __device__ constexpr int xbuf_elems(int log_l) { return xpad<PS>(1 << log_l); }

// Checked build (FCAS_CHECKED): the fitness kernels recompute each shared-memory, table and global
// index from its definition and range-test it; a failed test sets bit `bit` of this flag (read and
// cleared by the host after the launches) and the access is skipped. No trap, no fault.
#ifdef FCAS_CHECKED
static __device__ unsigned int g_index_checks;
__device__ __forceinline__ bool index_check(bool ok, int bit) {
    if (!ok) atomicOr(&g_index_checks, 1u << bit);
    return ok;
}
#define FCAS_CHECK(cond, bit) ::fcas::index_check((cond), (bit))
#else
#define FCAS_CHECK(cond, bit) true
#endif
enum IndexCheck { kCheckExchangeRead = 0, kCheckExchangeWrite = 1, kCheckTwiddle = 2, kCheckSpectrum = 3,
                  kCheckBasis = 4, kCheckInterWrite = 5, kCheckInterRead = 6 };

template <int S, typename C>
__device__ __forceinline__ void r16_dft4(C& a0, C& a1, C& a2, C& a3) {
    C t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = a1 - a3;
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = add_si<S>(t1, t3);
    a3 = sub_si<S>(t1, t3);
}

// the same transform with a2 given before its multiplication by S i (a twiddle of a quarter turn
// folded into the additions)
template <int S, typename C>
__device__ __forceinline__ void r16_dft4_a2si(C& a0, C& a1, C& a2, C& a3) {
    C t0 = add_si<S>(a0, a2), t1 = sub_si<S>(a0, a2), t2 = a1 + a3, t3 = a1 - a3;
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = add_si<S>(t1, t3);
    a3 = sub_si<S>(t1, t3);
}

// the same transform when a2 = a3 = 0 (the first layer of a column whose upper half is zero):
// a0 +- a1 and a0 +- i a1, without the additions of zero
template <int S, typename C>
__device__ __forceinline__ void r16_dft4_lowhalf(C& a0, C& a1, C& a2, C& a3) {
    const C x0 = a0, x1 = a1;
    a0 = x0 + x1;
    a2 = x0 - x1;
    a1 = add_si<S>(x0, x1);
    a3 = sub_si<S>(x0, x1);
}

// x * e^{S 2 pi i M / 16}
template <int S, int M, typename C>
__device__ __forceinline__ C rot16(C x) {
    using R = decltype(x.x);
    constexpr int m = M & 15;
    if constexpr (std::is_same<C, c32x2>::value) {
        return rot16_x2<S, m>(x);
    } else if constexpr (m == 0) {
        return x;
    } else if constexpr (m == 4) {
        return mul_si<S>(x);
    } else if constexpr (m == 8) {
        return mkc(-x.x, -x.y);
    } else if constexpr (m == 12) {
        return mul_si<-S>(x);
    } else {
        constexpr double kC[16] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                                   0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                                   -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173,
                                   0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613};
        constexpr double kS[16] = {0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613,
                                   1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                                   0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                                   -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173};
        if constexpr (m == 2 || m == 6 || m == 10 || m == 14) {
            // |c| = |s| = 1/sqrt 2: two multiplies instead of four
            const R k = (R)0.70710678118654752440;
            constexpr int sc = kC[m] > 0 ? 1 : -1, ss = S * kS[m] > 0 ? 1 : -1;
            return mkc(k * (sgn_mul<sc>(x.x) - sgn_mul<ss>(x.y)), k * (sgn_mul<ss>(x.x) + sgn_mul<sc>(x.y)));
        } else {
            const R c = (R)kC[m];
            const R s = (R)(S * kS[m]);
            return mkc(x.x * c - x.y * s, x.x * s + x.y * c);
        }
    }
}

// LH: a[R/2 ..] are zero (the first stage of a column whose upper half is zero)
template <int S, bool LH = false, typename C>
__device__ __forceinline__ void dft8(C (&a)[8]) {
    // n = 2 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle e^{S 2 pi i n2 k1 / 8}, DFT2 over n2
    C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    if constexpr (LH) {
        r16_dft4_lowhalf<S>(e0, e1, e2, e3);
        r16_dft4_lowhalf<S>(o0, o1, o2, o3);
    } else {
        r16_dft4<S>(e0, e1, e2, e3);
        r16_dft4<S>(o0, o1, o2, o3);
    }
    o1 = rot16<S, 2>(o1);
    o3 = rot16<S, 6>(o3);
    a[0] = e0 + o0;
    a[4] = e0 - o0;
    a[1] = e1 + o1;
    a[5] = e1 - o1;
    a[2] = add_si<S>(e2, o2);   // o2 e^{S 2 pi i 2 / 8} = S i o2
    a[6] = sub_si<S>(e2, o2);
    a[3] = e3 + o3;
    a[7] = e3 - o3;
}

template <int S, bool LH = false, typename C>
__device__ __forceinline__ void dft16(C (&a)[16]) {
    // n = 4 n1 + n2, k = k1 + 4 k2: DFT4 over n1 (for each n2), twiddle e^{S 2 pi i n2 k1 / 16},
    // DFT4 over n2 (for each k1)
    C y0[4] = {a[0], a[4], a[8], a[12]};
    C y1[4] = {a[1], a[5], a[9], a[13]};
    C y2[4] = {a[2], a[6], a[10], a[14]};
    C y3[4] = {a[3], a[7], a[11], a[15]};
    if constexpr (LH) {
        r16_dft4_lowhalf<S>(y0[0], y0[1], y0[2], y0[3]);
        r16_dft4_lowhalf<S>(y1[0], y1[1], y1[2], y1[3]);
        r16_dft4_lowhalf<S>(y2[0], y2[1], y2[2], y2[3]);
        r16_dft4_lowhalf<S>(y3[0], y3[1], y3[2], y3[3]);
    } else {
        r16_dft4<S>(y0[0], y0[1], y0[2], y0[3]);
        r16_dft4<S>(y1[0], y1[1], y1[2], y1[3]);
        r16_dft4<S>(y2[0], y2[1], y2[2], y2[3]);
        r16_dft4<S>(y3[0], y3[1], y3[2], y3[3]);
    }
    y1[1] = rot16<S, 1>(y1[1]);
    y1[2] = rot16<S, 2>(y1[2]);
    y1[3] = rot16<S, 3>(y1[3]);
    y2[1] = rot16<S, 2>(y2[1]);
    // y2[2] e^{S 2 pi i 4 / 16} = S i y2[2]: folded into its second-layer transform below
    y2[3] = rot16<S, 6>(y2[3]);
    y3[1] = rot16<S, 3>(y3[1]);
    y3[2] = rot16<S, 6>(y3[2]);
    y3[3] = rot16<S, 9>(y3[3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C b0 = y0[k1], b1 = y1[k1], b2 = y2[k1], b3 = y3[k1];
        if (k1 == 2) r16_dft4_a2si<S>(b0, b1, b2, b3);
        else r16_dft4<S>(b0, b1, b2, b3);
        a[k1] = b0;
        a[k1 + 4] = b1;
        a[k1 + 8] = b2;
        a[k1 + 12] = b3;
    }
}

template <int S, int R, bool LH = false, typename C>
__device__ __forceinline__ void dft_r(C (&a)[R]) {
    if constexpr (R == 16) dft16<S, LH>(a);
    else if constexpr (R == 8) dft8<S, LH>(a);
    else if constexpr (R == 4) r16_dft4<S>(a[0], a[1], a[2], a[3]);
    else if constexpr (R == 2) {
        C t = a[0] - a[1];
        a[0] = a[0] + a[1];
        a[1] = t;
    }
}

// LH (first stage only): the upper half of the input (v[V/2 ..]) is zero. TWL: the stage twiddles
// w^r (r < 4) and w^{4h} come from the table and the rest as one product each (instead of w and w^4
// loaded and the other powers formed by products); fewer instructions, a few more registers.
template <typename Real, int S, int LOG_L, int DONE, int MAXRB, bool PP, bool LH = false, bool TWL = false, int PS = 4>
__device__ __forceinline__ void fftr_stage(cplx<Real> (&v)[fftr_v(LOG_L, MAXRB)], cplx<Real>* buf0, int es, int j,
                                           const fft_tw<Real>* __restrict__ stw, int alt, int par0) {
    using C = cplx<Real>;
    using W = fft_tw<Real>;
    constexpr int L = 1 << LOG_L;
    constexpr int V = fftr_v(LOG_L, MAXRB);
    constexpr int G = L / V;
    constexpr int RB = fftr_radix_bits(LOG_L, DONE, MAXRB);
    constexpr int R = 1 << RB;
    constexpr int T = V / R;
    constexpr int NS = 1 << DONE;
    constexpr bool FIRST = DONE == 0;
    constexpr bool LAST = DONE + RB == LOG_L;
    constexpr int ST = DONE / MAXRB;
    if constexpr (!FIRST) {
        const cplx<Real>* buf = (PP && ((ST - 1 + par0) & 1)) ? buf0 + alt : buf0;
        if constexpr (G % (1 << PS) == 0) {
            // pad(j + q G) = pad(j) + q (G + G / 2^PS): one base address, constant offsets
            const C* rb = buf + xpad<PS>(j) * es;
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int e = xpad<PS>(j) + q * (G + (G >> PS));
                if (FCAS_CHECK(e == xpad<PS>(j + q * G) && e < xbuf_elems<PS>(LOG_L), kCheckExchangeRead))
                    v[q] = rb[q * (G + (G >> PS)) * es];
            }
        } else {
#pragma unroll
            for (int q = 0; q < V; ++q)
                if (FCAS_CHECK(xpad<PS>(j + q * G) < xbuf_elems<PS>(LOG_L), kCheckExchangeRead))
                    v[q] = buf[xpad<PS>(j + q * G) * es];
        }
    }
#pragma unroll
    for (int h = 0; h < T; ++h) {
        const int jj = j + h * G;
        C a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[h + r * T];
        if constexpr (NS > 1) {
            const int jm = jj & (NS - 1);
            const W* t = stw + (NS - 1) + jm;
            if constexpr (R >= 8 && TWL && !std::is_same<Real, ffloat>::value) {
                W wl[4], wh[R / 4];
                wl[0] = wh[0] = tw_one(W{});
#pragma unroll
                for (int r = 1; r < 4; ++r) {
                    wl[r] = wl[0];
                    if (FCAS_CHECK((NS - 1) + jm + (r - 1) * NS < L, kCheckTwiddle)) wl[r] = ldg_c(t + (r - 1) * NS);
                    if constexpr (S < 0) wl[r] = cconj(wl[r]);
                }
#pragma unroll
                for (int hi = 1; hi < R / 4; ++hi) {
                    wh[hi] = wh[0];
                    if (FCAS_CHECK((NS - 1) + jm + (4 * hi - 1) * NS < L, kCheckTwiddle))
                        wh[hi] = ldg_c(t + (4 * hi - 1) * NS);
                    if constexpr (S < 0) wh[hi] = cconj(wh[hi]);
                }
#pragma unroll
                for (int r = 1; r < 4; ++r) a[r] = cmul(a[r], wl[r]);
#pragma unroll
                for (int hi = 1; hi < R / 4; ++hi) {
                    a[4 * hi] = cmul(a[4 * hi], wh[hi]);
#pragma unroll
                    for (int r = 1; r < 4; ++r) a[4 * hi + r] = cmul(a[4 * hi + r], cmul(wh[hi], wl[r]));
                }
            } else if constexpr (R >= 8 && !std::is_same<Real, ffloat>::value) {
                // w^r for r = 1..R-1 from two table entries: w and w^4 (powers by products, <= 3 roundings);
                // the float-float form loads every power instead (a double-word product costs more
                // than a load)
                W w1 = tw_one(W{}), w4 = w1;
                if (FCAS_CHECK((NS - 1) + jm + 3 * NS < L, kCheckTwiddle)) {
                    w1 = ldg_c(t);
                    w4 = ldg_c(t + 3 * NS);
                }
                if constexpr (S < 0) {
                    w1 = cconj(w1);
                    w4 = cconj(w4);
                }
                const W w2 = cmul(w1, w1);
                const W w3 = cmul(w2, w1);
                a[1] = cmul(a[1], w1);
                a[2] = cmul(a[2], w2);
                a[3] = cmul(a[3], w3);
                W wb = w4;
#pragma unroll
                for (int hi = 1; hi < R / 4; ++hi) {
                    a[4 * hi] = cmul(a[4 * hi], wb);
                    a[4 * hi + 1] = cmul(a[4 * hi + 1], cmul(wb, w1));
                    a[4 * hi + 2] = cmul(a[4 * hi + 2], cmul(wb, w2));
                    a[4 * hi + 3] = cmul(a[4 * hi + 3], cmul(wb, w3));
                    if (hi + 1 < R / 4) wb = cmul(wb, w4);
                }
            } else {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    W w = tw_one(W{});
                    if (FCAS_CHECK((NS - 1) + (r - 1) * NS + jm < L, kCheckTwiddle)) w = ldg_c(t + (r - 1) * NS);
                    if constexpr (S < 0) w = cconj(w);
                    a[r] = cmul(a[r], w);
                }
            }
        }
        // with R = V (T = 1) the zero upper half of the first stage is the upper half of a[]
        dft_r<S, R, LH && FIRST && T == 1 && R >= 8>(a);
#pragma unroll
        for (int r = 0; r < R; ++r) v[h + r * T] = a[r];
    }
    if constexpr (!LAST) {
        if constexpr (!PP) __syncthreads();
        cplx<Real>* buf = (PP && ((ST + par0) & 1)) ? buf0 + alt : buf0;
#pragma unroll
        for (int h = 0; h < T; ++h) {
            const int jj = j + h * G;
            const int dst = (jj / NS) * NS * R + (jj & (NS - 1));
            // pad(dst + r NS) = pad(dst) + r NS + (r NS >> PS) when adding r NS to dst never carries
            // into a new group of 2^PS differently from r NS itself: NS a multiple of 2^PS, or NS
            // dividing 2^PS with NS R a multiple of 2^PS (dst mod 2^PS < NS), or PS = 4, NS = 1 and
            // R = 8 (dst mod 16 in {0, 8})
            constexpr int GP = 1 << PS;
            if constexpr (NS % GP == 0 || (GP % NS == 0 && (NS * R) % GP == 0) || (PS == 4 && NS == 1 && R == 8)) {
                C* wb = buf + xpad<PS>(dst) * es;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int e = xpad<PS>(dst) + r * NS + ((r * NS) >> PS);
                    if (FCAS_CHECK(e == xpad<PS>(dst + r * NS) && e < xbuf_elems<PS>(LOG_L), kCheckExchangeWrite))
                        wb[(r * NS + ((r * NS) >> PS)) * es] = v[h + r * T];
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (FCAS_CHECK(xpad<PS>(dst + r * NS) < xbuf_elems<PS>(LOG_L), kCheckExchangeWrite))
                        buf[xpad<PS>(dst + r * NS) * es] = v[h + r * T];
            }
        }
        __syncthreads();
    }
}

template <typename Real, int S, int LOG_L, int MAXRB, bool PP = false, int DONE = 0, bool LH = false, bool TWL = false,
          int PS = 4>
__device__ __forceinline__ void fftr(cplx<Real> (&v)[fftr_v(LOG_L, MAXRB)], cplx<Real>* buf, int es, int j,
                                     const fft_tw<Real>* __restrict__ stw, int alt = 0, int par0 = 0) {
    if constexpr (DONE < LOG_L) {
        fftr_stage<Real, S, LOG_L, DONE, MAXRB, PP, LH, TWL, PS>(v, buf, es, j, stw, alt, par0);
        fftr<Real, S, LOG_L, MAXRB, PP, DONE + fftr_radix_bits(LOG_L, DONE, MAXRB), false, TWL, PS>(v, buf, es, j, stw,
                                                                                                  alt, par0);
    }
}

template <typename Real, int S, int LOG_L, bool PP = false>
__device__ __forceinline__ void fft16(cplx<Real> (&v)[fft16_v(LOG_L)], cplx<Real>* buf, int es, int j,
                                      const fft_tw<Real>* __restrict__ stw, int alt = 0, int par0 = 0) {
    fftr<Real, S, LOG_L, 4, PP>(v, buf, es, j, stw, alt, par0);
}

}  // namespace fcas
