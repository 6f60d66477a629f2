// Instantiations of the persistent two-pass launch (fft_fused.cuh) for the
// FP32 path: one CTA shape per split, both passes at the same thread count.
#include "fft_fused.cuh"

namespace fstat {

namespace {
constexpr int key(int l1, int l2) { return l1 * 16 + l2; }
}  // namespace

bool fused_supported(int log2n1, int log2n2) {
  switch (key(log2n1, log2n2)) {
    case key(9, 9): case key(9, 10): case key(10, 10): case key(10, 11): case key(10, 12): case key(11, 12):
    case key(12, 12):
      return true;
    default:
      return false;
  }
}

cudaError_t launch_fused_f32(int log2n1, int log2n2, const FusedArgs& a, cudaStream_t st) {
  // template arguments: pass A length (n2), columns per CTA, schedule;
  // pass B length (n1), rows per CTA, schedule (one buffer, bulk copies)
  switch (key(log2n1, log2n2)) {
    case key(9, 9): return fft::run_fused<512, 4, 6, 512, 4, 6>(a, st);
    case key(9, 10): return fft::run_fused<1024, 4, 6, 512, 4, 6>(a, st);
    case key(10, 10): return fft::run_fused<1024, 4, 6, 1024, 4, 6>(a, st);
    case key(10, 11): return fft::run_fused<2048, 2, 6, 1024, 4, 6>(a, st);
    case key(10, 12): return fft::run_fused<4096, 1, 6, 1024, 4, 6>(a, st);
    case key(11, 12): return fft::run_fused<4096, 1, 6, 2048, 2, 6>(a, st);
    case key(12, 12): return fft::run_fused<4096, 2, 6, 4096, 2, 6>(a, st);
    default: return cudaErrorInvalidConfiguration;
  }
}

}  // namespace fstat
