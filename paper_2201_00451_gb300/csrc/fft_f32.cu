// FP32 (mixed-precision path) instantiations of the FFT passes.
#include "fft_impl.cuh"

namespace fstat {

cudaError_t launch_pass_a_f32(int log2_n2, const void* G, int64_t lc, int64_t n, int n1, int log2N,
                              const TmplCoef* coef, void* Z, cudaStream_t st) {
  return fft::dispatch_a<float>(log2_n2, G, lc, n, n1, log2N, coef, Z, st);
}

cudaError_t launch_pass_b_f32(int log2_n1, const void* Z, int n2, const SkyConst* sky, float* out,
                              cudaStream_t st) {
  return fft::dispatch_b<float>(log2_n1, Z, n2, sky, out, st);
}

}  // namespace fstat
