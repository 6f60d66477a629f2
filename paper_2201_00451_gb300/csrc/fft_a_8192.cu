// FP32 instantiations of FFT pass A for 8192-point columns (radix 16 x 16 x
// 16 x 2, or radix-8 first; the input staged in shared memory of its own
// with schedule 16), used by the split 2048 x 8192 of n_fft = 2^24:
// its pass B then transforms 2048-point rows four at a time.  Kept apart
// from fft_a_f32.cu so the two compile in parallel.
#include "fft_impl.cuh"

namespace fstat {
namespace fft {

cudaError_t pick_a_8192(int ca, int v, const void* G, int64_t lc, int64_t n, int n1, const void* twA,
                        const TmplCoef* coef, void* Z, int* err, int wait_limit, cudaStream_t st, int res) {
  return pick_a<float, 8192>(ca, v, G, lc, n, n1, twA, coef, Z, err, wait_limit, st, res);
}

}  // namespace fft
}  // namespace fstat
