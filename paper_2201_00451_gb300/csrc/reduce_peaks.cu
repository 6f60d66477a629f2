// fstat_reduce_peaks: the peaks reduction of fstat_compute_peaks applied to
// 2F rows already in device memory (a semi-coherent sum, or any dense
// output): threshold crossings and band maxima.  Each CTA takes 4096
// consecutive bins of one row, each thread 16 consecutive bins, and runs
// the same epilogue as the last FFT pass in peaks mode (bin f of the CTA's
// run is start + f).
#include "fft_impl.cuh"
#include "reduce_peaks.cuh"

namespace fstat {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedPer = 16;                       // bins per thread
constexpr int kRedRun = kRedThreads * kRedPer;    // bins per CTA

__global__ void __launch_bounds__(kRedThreads)
k_reduce_peaks(const float* __restrict__ twoF, int64_t n_bins, PeakArgs pk, int64_t row0, int64_t key_stride) {
  const int64_t row = blockIdx.y;
  const int64_t start = (int64_t)blockIdx.x * kRedRun;
  PeakArgs a = pk;
  a.tmpl = pk.tmpl + row0 + row;
  if (a.band_key) a.band_key = pk.band_key + row * key_stride;
  fft::peak_epilogue<1, kRedPer>(twoF + row * n_bins + start, (int)start, 1, a, nullptr);
}

}  // namespace

cudaError_t launch_reduce_peaks(const float* twoF, int64_t n_rows, int64_t n_bins, const PeakArgs& pk,
                                int64_t key_stride, cudaStream_t st) {
  if (n_bins % kRedRun) return cudaErrorInvalidValue;
  for (int64_t r0 = 0; r0 < n_rows; r0 += 65535) {
    const int64_t rows = n_rows - r0 < 65535 ? n_rows - r0 : 65535;
    PeakArgs a = pk;
    if (a.band_key) a.band_key = pk.band_key + r0 * key_stride;
    const dim3 grid((unsigned)(n_bins / kRedRun), (unsigned)rows);
    k_reduce_peaks<<<grid, kRedThreads, 0, st>>>(twoF + r0 * n_bins, n_bins, a, r0, key_stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fstat
