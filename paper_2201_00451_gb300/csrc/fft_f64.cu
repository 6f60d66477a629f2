// FP64 (comparison path) instantiations of the FFT passes.
#include "fft_impl.cuh"

namespace fstat {

cudaError_t launch_pass_a_f64(int log2_n2, int ca, int va, const void* G, int64_t lc, int64_t n, int n1,
                              const void* twA, const TmplCoef* coef, void* Z, cudaStream_t st, int res, int* err,
                              int wait_limit) {
  return fft::dispatch_a<double>(log2_n2, ca, va, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
}

cudaError_t launch_pass_b_f64(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                              const SkyConst* sky, float* out, cudaStream_t st, const PeakArgs* pk,
                              int res, int* err, int wait_limit) {
  if (pk) {
    PeakArgs a = *pk;
    if (!a.err) a.err = err;
    set_wait(a, wait_limit);
    return launch_pass_b_peak_f64(log2_n1, cb, vb, Z, n2, twB, sky, a, st, res);
  }
  PeakArgs a{};
  a.err = err;
  set_wait(a, wait_limit);
  return fft::dispatch_b<double, fft::kStore>(log2_n1, cb, vb, Z, n2, twB, sky, out, a, st, res);
}

}  // namespace fstat
