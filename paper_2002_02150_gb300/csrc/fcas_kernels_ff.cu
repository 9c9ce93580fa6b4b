// The float-float form of the two FFT passes (fcas_passes.cuh instantiated with Real = ffloat):
// binary64-class accuracy from the FP32 units, the phase generated in binary64.
#include "fcas_passes.cuh"

namespace fcas {

template cudaError_t launch_pass_a<ffloat>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, void*,
                                           cudaStream_t);
template cudaError_t launch_pass_b<ffloat>(const FitnessPlan&, const ParticleParams*, int64_t, int64_t, const void*,
                                           Partial*, cudaStream_t);

// index checks of this translation unit's kernels (checked build; 0 otherwise)
unsigned int take_index_checks_ff(cudaStream_t s) {
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

}  // namespace fcas
