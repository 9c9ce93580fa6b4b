// Block-level Stockham FFT used by both passes of the length-N transform over t_c.
//
// A transform of length L = 2^LOG_L is held by G = L / V threads, thread j owning the V values at
// positions j + q G (q = 0..V-1) on entry and on exit (natural order in and out). Each stage of
// radix R (4, or 2 for a last odd bit) performs the Stockham self-sorting step: task jj reads
// x[jj + r L/R], multiplies by e^{S 2 pi i r (jj mod Ns) / (Ns R)}, applies the R-point DFT and
// writes to (jj / Ns) Ns R + (jj mod Ns) + r Ns. Stages are separated by a shared-memory exchange;
// the first stage takes its inputs from registers and the last one leaves its outputs there.
// S = +1 computes sum_k x[k] e^{+2 pi i k t / L}, S = -1 the forward transform.
#pragma once

#include "fcas_internal.cuh"

namespace fcas {

template <int S, typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = a1 - a3;
    C it3 = mul_si<S>(t3);
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = t1 + it3;
    a3 = t1 - it3;
}

template <typename C>
__device__ __forceinline__ void dft2(C& a0, C& a1) {
    C t = a0 - a1;
    a0 = a0 + a1;
    a1 = t;
}

// Twiddle e^{S 2 pi i m / L} from a table of e^{2 pi i m' / TWL} (TWL = L << tw_shift).
template <int S, typename C>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, int m, int tw_shift) {
    C w = __ldg(tw + (m << tw_shift));
    return S > 0 ? w : cconj(w);
}

template <typename Real, int S, int LOG_L, int V, int RB, int DONE>
__device__ __forceinline__ void fft_stage(cplx<Real> (&v)[V], cplx<Real>* buf, int es, int j,
                                          const cplx<Real>* __restrict__ tw, int tw_shift) {
    using C = cplx<Real>;
    constexpr int L = 1 << LOG_L;
    constexpr int G = L / V;
    constexpr int R = 1 << RB;
    constexpr int T = V / R;          // tasks per thread
    constexpr int NS = 1 << DONE;
    constexpr bool FIRST = DONE == 0;
    constexpr bool LAST = DONE + RB == LOG_L;
    if constexpr (!FIRST) {
#pragma unroll
        for (int q = 0; q < V; ++q) v[q] = buf[(j + q * G) * es];
    }
#pragma unroll
    for (int h = 0; h < T; ++h) {
        const int jj = j + h * G;
        if constexpr (NS > 1) {
            const int jm = jj & (NS - 1);
            constexpr int STEP = L / (NS * R);
#pragma unroll
            for (int r = 1; r < R; ++r) v[h + r * T] = cmul(v[h + r * T], twiddle<S>(tw, r * jm * STEP, tw_shift));
        }
        if constexpr (R == 4) dft4<S>(v[h], v[h + T], v[h + 2 * T], v[h + 3 * T]);
        else dft2(v[h], v[h + T]);
    }
    if constexpr (!LAST) {
        __syncthreads();
#pragma unroll
        for (int h = 0; h < T; ++h) {
            const int jj = j + h * G;
            const int dst = (jj / NS) * NS * R + (jj & (NS - 1));
#pragma unroll
            for (int r = 0; r < R; ++r) buf[(dst + r * NS) * es] = v[h + r * T];
        }
        __syncthreads();
    }
}

template <typename Real, int S, int LOG_L, int V, int DONE = 0>
__device__ __forceinline__ void block_fft(cplx<Real> (&v)[V], cplx<Real>* buf, int es, int j,
                                          const cplx<Real>* __restrict__ tw, int tw_shift) {
    constexpr int REM = LOG_L - DONE;
    if constexpr (REM > 0) {
        constexpr int RB = REM >= 2 ? 2 : 1;
        fft_stage<Real, S, LOG_L, V, RB, DONE>(v, buf, es, j, tw, tw_shift);
        block_fft<Real, S, LOG_L, V, DONE + RB>(v, buf, es, j, tw, tw_shift);
    }
}

}  // namespace fcas
