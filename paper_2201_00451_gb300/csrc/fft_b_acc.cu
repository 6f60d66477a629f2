// Pass B in accumulate mode (fstat_semicoherent): the same transform as the
// dense pass, with each segment's 2F added to the output row at a bin offset.
#include "fft_impl.cuh"

namespace fstat {

cudaError_t launch_pass_b_acc_f32(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                                  const SkyConst* sky, float* out, int shift, cudaStream_t st, int res,
                                  int* err, int wait_limit) {
  PeakArgs a{};
  a.shift = shift;
  a.err = err;
  set_wait(a, wait_limit);
  return fft::dispatch_b<float, fft::kAccumulate>(log2_n1, cb, vb, Z, n2, twB, sky, out, a, st, res);
}

cudaError_t launch_pass_b_acc_f64(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                                  const SkyConst* sky, float* out, int shift, cudaStream_t st, int res,
                                  int* err, int wait_limit) {
  PeakArgs a{};
  a.shift = shift;
  a.err = err;
  set_wait(a, wait_limit);
  return fft::dispatch_b<double, fft::kAccumulate>(log2_n1, cb, vb, Z, n2, twB, sky, out, a, st, res);
}

}  // namespace fstat
