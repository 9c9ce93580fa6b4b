// Per-particle diagnostics outside the fitness path: the condition number of the antenna-pattern
// matrix (Sec. V).
#include "fcas_diag.cuh"

namespace fcas {

// ------------------------------------------------------------------------------------------
// Condition number of the antenna-pattern matrix F(alpha, delta, psi) (Sec. V): the ratio of the
// singular values of the (D, 2) matrix, from the eigenvalues of F^T F (independent of psi).
// ------------------------------------------------------------------------------------------
__global__ void condition_kernel(const double* __restrict__ theta, int64_t n, const double* __restrict__ det9,
                                 int n_det, double* __restrict__ kappa) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double alpha = theta[4 * p + 0], delta = theta[4 * p + 1];
    if (!(isfinite(alpha) && isfinite(delta))) {
        kappa[p] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    double sa, ca, sd, cd;
    sincos(alpha, &sa, &ca);
    sincos(delta, &sd, &cd);
    const double bx[3] = {sa, -ca, 0.0};
    const double by[3] = {-sd * ca, -sd * sa, cd};
    double a = 0.0, b = 0.0, c = 0.0;   // F^T F = [[a, b], [b, c]]
    for (int i = 0; i < n_det; ++i) {
        const double* d = det9 + 9 * i;
        const double xX = d[3] * bx[0] + d[4] * bx[1] + d[5] * bx[2];
        const double xY = d[3] * by[0] + d[4] * by[1] + d[5] * by[2];
        const double yX = d[6] * bx[0] + d[7] * bx[1] + d[8] * bx[2];
        const double yY = d[6] * by[0] + d[7] * by[1] + d[8] * by[2];
        const double fp = 0.5 * (xX * xX - xY * xY - yX * yX + yY * yY);
        const double fx = xX * xY - yX * yY;
        a += fp * fp;
        b += fp * fx;
        c += fx * fx;
    }
    const double det = a * c - b * b, tr = a + c;
    if (det < kRank1Rtol * (0.5 * tr) * (0.5 * tr)) {     // numerically rank one (the rule used for G)
        kappa[p] = __longlong_as_double(0x7ff0000000000000LL);
        return;
    }
    const double hi = 0.5 * tr + sqrt(0.25 * (a - c) * (a - c) + b * b);
    kappa[p] = sqrt(hi / (det / hi));                      // larger / smaller eigenvalue of F^T F
}

cudaError_t launch_condition(const double* theta, int64_t n, const double* det9, int n_det, double* kappa,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int threads = 128;
    condition_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(theta, n, det9, n_det, kappa);
    return cudaGetLastError();
}

}  // namespace fcas
