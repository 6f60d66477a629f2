// Pass B in peaks mode (fstat_compute_peaks): the same transform as the
// dense pass, with 2F reduced in the kernel to a threshold-crossing list and
// per-band maxima.  Both precisions live here so the dense translation
// units keep their build time.
#include "fft_impl.cuh"

namespace fstat {

cudaError_t launch_pass_b_peak_f32(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                                   const SkyConst* sky, const PeakArgs& pk, cudaStream_t st, int res) {
  return fft::dispatch_b<float, fft::kPeaks>(log2_n1, cb, vb, Z, n2, twB, sky, nullptr, pk, st, res);
}

cudaError_t launch_pass_b_peak_f64(int log2_n1, int cb, int vb, const void* Z, int n2, const void* twB,
                                   const SkyConst* sky, const PeakArgs& pk, cudaStream_t st, int res) {
  return fft::dispatch_b<double, fft::kPeaks>(log2_n1, cb, vb, Z, n2, twB, sky, nullptr, pk, st, res);
}

namespace {

__global__ void k_band_decode(const unsigned long long* __restrict__ keys, int64_t count,
                              float* __restrict__ band_max, int32_t* __restrict__ band_bin) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[i];
    unsigned u = (unsigned)(k >> 32);
    u ^= (u & 0x80000000u) ? 0x80000000u : 0xffffffffu;   // inverse of band_key's map
    band_max[i] = __uint_as_float(u);
    if (band_bin) band_bin[i] = (int32_t)(0xffffffffu - (unsigned)(k & 0xffffffffu));
  }
}

}  // namespace

cudaError_t launch_band_decode(const unsigned long long* keys, int64_t count, float* band_max,
                               int32_t* band_bin, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t want = (count + threads - 1) / threads;
  const int grid = (int)(want < 4096 ? want : 4096);
  k_band_decode<<<grid, threads, 0, st>>>(keys, count, band_max, band_bin);
  return cudaGetLastError();
}

}  // namespace fstat
