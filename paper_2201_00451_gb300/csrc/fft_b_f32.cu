// FP32 (mixed-precision path) instantiations of FFT pass B.
#include "fft_impl.cuh"

namespace fstat {

cudaError_t launch_pass_b_f32(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                              const SkyConst* sky, float* out, cudaStream_t st, const PeakArgs* pk,
                              int res, int* err, int wait_limit) {
  if (pk) {
    PeakArgs a = *pk;
    if (!a.err) a.err = err;
    set_wait(a, wait_limit);
    return launch_pass_b_peak_f32(log2_n1, cb, vb, Z, n2, twB, sky, a, st, res);
  }
  PeakArgs a{};
  a.err = err;
  set_wait(a, wait_limit);
  return fft::dispatch_b<float, fft::kStore>(log2_n1, cb, vb, Z, n2, twB, sky, out, a, st, res);
}

}  // namespace fstat
