// Machine peaks for the roofline figures the benchmark reports: the FP32
// and FP64 fused multiply-add rates of the CUDA cores, measured on the
// current device with a kernel of independent FMA chains on every SM (the
// FFT passes are bound by FP32 instruction issue, the per-sky timing by
// the FP64 pipe, so both rates are denominators the library's kernels are
// judged against).  Not part of the F-statistic computation.

#include "fstat_internal.cuh"

namespace fstat {
namespace {

constexpr int kChains = 8;        // independent FMA chains per thread
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_peak(T* __restrict__ sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a value the chains never reach keeps them live without a store per thread
  if (s == (T)-1.2345e30) sink[blockIdx.x] = s;
}

template <typename T>
int probe(int64_t iters, double* tflops, double* ms_out, cudaStream_t st) {
  const int sms = device_sm_count();
  const int blocks = sms * (2048 / kProbeThreads);
  T* sink = nullptr;  // never written (see the kernel)
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FSTAT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return FSTAT_ERR_CUDA; }
  // a, b keep the chains bounded (|x| stays below b / (1 - a))
  const T a = (T)0.999999, b = (T)1e-6;
  k_fma_peak<T><<<blocks, kProbeThreads, 0, st>>>(sink, (int)iters, a, b);  // warm-up
  cudaEventRecord(e0, st);
  k_fma_peak<T><<<blocks, kProbeThreads, 0, st>>>(sink, (int)iters, a, b);
  cudaEventRecord(e1, st);
  int rc = FSTAT_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = FSTAT_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kProbeThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return FSTAT_OK;
}

}  // namespace
}  // namespace fstat

using namespace fstat;

extern "C" int fstat_probe_fma(int precision, int64_t iters, double* tflops, double* ms, void* stream) {
  if (!tflops || iters < 1 || iters > (int64_t)1 << 30 || (precision != FSTAT_MIXED && precision != FSTAT_FP64))
    return FSTAT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == FSTAT_FP64 ? probe<double>(iters, tflops, ms, st) : probe<float>(iters, tflops, ms, st);
}
