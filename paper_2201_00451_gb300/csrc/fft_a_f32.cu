// FP32 (mixed-precision path) instantiations of FFT pass A.
#include "fft_impl.cuh"

namespace fstat {

cudaError_t launch_pass_a_f32(int log2_n2, int ca, int va, const void* G, int64_t lc, int64_t n, int n1,
                              const void* twA, const TmplCoef* coef, void* Z, cudaStream_t st, int res, int* err,
                              int wait_limit) {
  return fft::dispatch_a<float>(log2_n2, ca, va, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
}

namespace {
template <typename T, int L> int default_ca() { return fft::Shape<T, L, 0>::CA_DEF; }
template <typename T, int L> int default_cb() { return fft::Shape<T, L, 0>::CB_DEF; }
template <typename T, int L> int default_c(bool pass_b) { return pass_b ? default_cb<T, L>() : default_ca<T, L>(); }
template <typename T> int default_c_len(int log2_len, bool pass_b) {
  switch (log2_len) {
    case 5: return default_c<T, 32>(pass_b);
    case 6: return default_c<T, 64>(pass_b);
    case 7: return default_c<T, 128>(pass_b);
    case 8: return default_c<T, 256>(pass_b);
    case 9: return default_c<T, 512>(pass_b);
    case 10: return default_c<T, 1024>(pass_b);
    case 11: return default_c<T, 2048>(pass_b);
    case 12: return default_c<T, 4096>(pass_b);
    case 13: return pass_b ? 0 : 1;  // 8192-point columns: one per CTA
    default: return 0;
  }
}
}  // namespace

// Columns (pass A, pass_b = 0) or rows (pass B) per CTA that shape 0 stands
// for at a pass length 2^log2_len.
int fft_default_c(int log2_len, int pass_b, int precision) {
  return precision == FSTAT_FP64 ? default_c_len<double>(log2_len, pass_b != 0)
                                 : default_c_len<float>(log2_len, pass_b != 0);
}

}  // namespace fstat
