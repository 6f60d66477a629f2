// FP32 (mixed-precision path) instantiations of FFT pass A.
#include "fft_impl.cuh"

namespace fstat {

cudaError_t launch_pass_a_f32(int log2_n2, int ca, int va, const void* G, int64_t lc, int64_t n, int n1,
                              const void* twA, const void* hi, const void* lo, int h, const TmplCoef* coef,
                              void* Z, cudaStream_t st) {
  return fft::dispatch_a<float>(log2_n2, ca, va, G, lc, n, n1, twA, hi, lo, h, coef, Z, st);
}

}  // namespace fstat
