// Machine peaks for the roofline figures the benchmark reports: the FP32
// and FP64 fused multiply-add rates of the CUDA cores, measured on the
// current device with a kernel of independent FMA chains on every SM (the
// FFT passes are bound by FP32 instruction issue, the per-sky timing by
// the FP64 pipe, so both rates are denominators the library's kernels are
// judged against).  Not part of the F-statistic computation.

#include "fft_impl.cuh"  // the passes' radix-16 butterflies (fft::dft16)

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

namespace fstat {
namespace {

// ---------------------------------------------------------------------------
// Radix-16 DFT stage two ways, for the choice between CUDA cores and tensor
// cores in the FFT passes (X_m = sum_s x_s exp(-2 pi i m s / 16), the first
// radix-16 stage of every column and row transform):
//   method 0: the FFT passes' own butterflies (fft::dft16 on Fa/Fb pairs in
//             registers, CUDA cores);
//   method 1: the same stage as a matrix product on the tensor cores: the
//             real 32 x 32 form of the 16-point DFT matrix times 32 x 8
//             column blocks (mma.sync m16n8k8, TF32), with each operand split
//             into a TF32 head and a TF32 tail and three products (head*head +
//             head*tail + tail*head) so that the result keeps FP32-level
//             accuracy (one TF32 product alone carries ~1e-3 relative error,
//             the size of the 2F tolerance).
// Each CTA stages its 16-point vectors in shared memory, runs the stage
// `reps` times in place (the global traffic is paid once), and writes them
// back.  Data layout (global and shared): method 0 float4 pairs
// (a.re, a.im, b.re, b.im) [s][vector]; method 1 floats [vector][k], k < 16
// the real parts, k >= 16 the imaginary parts.  The vectors per CTA are the
// same for both methods (2 x 256: Fa and Fb of 256 butterflies).
constexpr int kDftVec = 512;  // 16-point complex vectors per CTA

__global__ void __launch_bounds__(256) k_dft16_simt(const float4* __restrict__ in, float4* __restrict__ out,
                                                    int reps) {
  extern __shared__ float4 buf[];  // [16][256]
  const int t = threadIdx.x;
  const float4* src = in + (int64_t)blockIdx.x * 16 * 256;
#pragma unroll
  for (int s = 0; s < 16; ++s) buf[s * 256 + t] = src[s * 256 + t];
  for (int r = 0; r < reps; ++r) {
    Pair<float> v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = pload(buf + s * 256 + t);
    fft::dft16(v);
#pragma unroll
    for (int s = 0; s < 16; ++s) pstore(buf + s * 256 + t, v[s]);
  }
  float4* dst = out + (int64_t)blockIdx.x * 16 * 256;
#pragma unroll
  for (int s = 0; s < 16; ++s) dst[s * 256 + t] = buf[s * 256 + t];
}

__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// real 32 x 32 form of the 16-point DFT matrix: rows m < 16 give Re X_m,
// m >= 16 Im X_(m-16); columns k < 16 take Re x_k, k >= 16 Im x_(k-16)
__device__ __forceinline__ float dft_real(int m, int k) {
  const int mm = m & 15, kk = k & 15;
  double sn, cs;
  sincospi(-2.0 * (double)((mm * kk) & 15) / 16.0, &sn, &cs);  // exp(-2 pi i m k / 16)
  if (m < 16) return (float)(k < 16 ? cs : -sn);
  return (float)(k < 16 ? sn : cs);
}

__global__ void __launch_bounds__(256) k_dft16_mma(const float* __restrict__ in, float* __restrict__ out, int reps) {
  extern __shared__ float bufm[];  // [vector][k], row pitch 33 floats (no bank conflicts)
  float* buf = bufm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const float* src = in + (int64_t)blockIdx.x * kDftVec * 32;
  for (int i = threadIdx.x; i < kDftVec * 32; i += 256) buf[(i >> 5) * 33 + (i & 31)] = src[i];
  // the DFT matrix as A fragments (2 row tiles x 4 k steps), head and tail
  unsigned ah[2][4][4], al[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = mt * 16 + g + (q & 1) * 8, k = ks * 8 + tg + (q >> 1) * 4;
        const float w = dft_real(m, k);
        ah[mt][ks][q] = to_tf32(w);
        al[mt][ks][q] = to_tf32(w - __uint_as_float(ah[mt][ks][q]));
      }
  __syncthreads();
  // each warp owns 64 vectors: 8 column blocks of 8
  float* wb = buf + warp * 64 * 33;
  for (int r = 0; r < reps; ++r) {
#pragma unroll 1
    for (int nt = 0; nt < 8; ++nt) {
      float* col = wb + (nt * 8 + g) * 33;  // this lane's B column (vector)
      unsigned bh[4][2], bl[4][2];
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float x = col[ks * 8 + tg + q * 4];
          bh[ks][q] = to_tf32(x);
          bl[ks][q] = to_tf32(x - __uint_as_float(bh[ks][q]));
        }
      float d[2][4] = {};
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          mma_tf32(d[mt], al[mt][ks], bh[ks]);
          mma_tf32(d[mt], ah[mt][ks], bl[ks]);
          mma_tf32(d[mt], ah[mt][ks], bh[ks]);
        }
      __syncwarp();  // every lane has read its operands before the results overwrite them
      // D fragment: rows m = mt*16 + g (+8), columns n = 2 tg (+1) of the block
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int m = mt * 16 + g + (q >> 1) * 8, n = nt * 8 + 2 * tg + (q & 1);
          wb[n * 33 + m] = d[mt][q];
        }
      __syncwarp();
    }
  }
  __syncthreads();
  float* dst = out + (int64_t)blockIdx.x * kDftVec * 32;
  for (int i = threadIdx.x; i < kDftVec * 32; i += 256) dst[i] = buf[(i >> 5) * 33 + (i & 31)];
}

}  // namespace
}  // namespace fstat

extern "C" int fstat_probe_dft16(int method, const void* in, void* out, int64_t n_vectors, int reps, double* ms,
                                 void* stream) {
  if (!in || !out || !ms || (method != 0 && method != 1) || n_vectors < kDftVec || n_vectors % kDftVec ||
      reps < 1 || n_vectors / kDftVec > INT32_MAX)
    return FSTAT_ERR_INVALID_ARG;
  if (((uintptr_t)in | (uintptr_t)out) & 15) return FSTAT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = (int)(n_vectors / kDftVec);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FSTAT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return FSTAT_ERR_CUDA; }
  constexpr size_t kSimtSmem = 16 * 256 * sizeof(float4), kMmaSmem = kDftVec * 33 * sizeof(float);
  if (cudaFuncSetAttribute(k_dft16_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSimtSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_dft16_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmaSmem) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return FSTAT_ERR_CUDA;
  }
  auto launch = [&] {
    if (method == 0) k_dft16_simt<<<blocks, 256, kSimtSmem, st>>>((const float4*)in, (float4*)out, reps);
    else k_dft16_mma<<<blocks, 256, kMmaSmem, st>>>((const float*)in, (float*)out, reps);
  };
  launch();  // warm-up
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  float t = 0.f;
  int rc = FSTAT_OK;
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
    rc = FSTAT_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t;
  return rc;
}
