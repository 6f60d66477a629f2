// Step (ii) of Sec. 3 from short Fourier transforms (fstat_set_sfts): per
// SFT s the band of B bins around f_h is inverse-transformed to B samples
// at dt = T_sft / B, rotated by exp(-2 pi i f_h t_s) and scaled by 1/M:
//
//   x_h[s B + m] = exp(-2 pi i f_h t_s) / M * sum_{i=0}^{B-1} X_s[i] exp(2 pi i (i - B/2) m / B)
//
// (column i of the band holds SFT bin q_h - B/2 + i).  B need not be a
// power of two, so the transform is the direct sum: one CTA per (SFT,
// block of output samples) stages the SFT's bins and the B roots of unity
// in shared memory, and each thread accumulates kSftOut outputs, advancing
// every root index (i - B/2) m mod B by m per bin (exact integer
// reduction).  FP32 accumulation for mixed plans, FP64 for FP64 plans.

#include <math.h>

#include "fstat_internal.cuh"
#include "sft.cuh"

namespace fstat {

namespace {

constexpr int kSftThreads = 256;
constexpr int kSftOut = 4;  // output samples per thread

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

// exp(2 pi i j / B), j < B, computed in FP64
template <typename T>
__global__ void k_sft_roots(int64_t B, typename C2<T>::type* __restrict__ w) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < B; j += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)j / (double)B, &s, &c);
    w[j] = {(T)c, (T)s};
  }
}

template <typename T, typename TIn>
__global__ void __launch_bounds__(kSftThreads)
k_sft_to_xh(const TIn* __restrict__ bins, const typename C2<T>::type* __restrict__ roots, int B,
            double f_het, double t_start, double t_sft, double inv_m, typename C2<T>::type* __restrict__ xh) {
  using V = typename C2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sx = reinterpret_cast<V*>(smem_raw);  // the SFT's bins
  V* sw = sx + B;                          // roots of unity
  const int s = blockIdx.y;
  const TIn* src = bins + (int64_t)s * B;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const TIn v = src[i];
    sx[i] = {(T)v.x, (T)v.y};
    sw[i] = roots[i];
  }
  __syncthreads();
  // outputs m_r = base + r * blockDim.x of this thread
  const int base = blockIdx.x * (kSftThreads * kSftOut) + threadIdx.x;
  int m[kSftOut], j[kSftOut];
  T ar[kSftOut], ai[kSftOut];
#pragma unroll
  for (int r = 0; r < kSftOut; ++r) {
    m[r] = base + r * kSftThreads;
    const int mm = m[r] < B ? m[r] : 0;
    // root index for bin i = 0: (-B/2) m mod B
    j[r] = (int)(((int64_t)(B - B / 2) * mm) % B);
    ar[r] = 0;
    ai[r] = 0;
  }
  for (int i = 0; i < B; ++i) {
    const V x = sx[i];
#pragma unroll
    for (int r = 0; r < kSftOut; ++r) {
      const V w = sw[j[r]];
      ar[r] += x.x * w.x - x.y * w.y;
      ai[r] += x.x * w.y + x.y * w.x;
      j[r] += m[r] < B ? m[r] : 0;
      if (j[r] >= B) j[r] -= B;
    }
  }
  // exp(-2 pi i f_h t_s) / M with f_h t_s reduced mod 1 in FP64
  const double t_s = t_start + (double)s * t_sft;
  double ph = f_het * t_s;
  ph -= floor(ph);
  double sn, cs;
  sincospi(2.0 * ph, &sn, &cs);
  const T rc = (T)(cs * inv_m), rs = (T)(-sn * inv_m);
#pragma unroll
  for (int r = 0; r < kSftOut; ++r) {
    if (m[r] >= B) continue;
    xh[(int64_t)s * B + m[r]] = {ar[r] * rc - ai[r] * rs, ar[r] * rs + ai[r] * rc};
  }
}

template <typename T, typename TIn>
cudaError_t run_sft(const void* bins, int64_t n_sft, int B, double f_het, double t_start, double t_sft,
                    int64_t m_raw, void* roots, void* xh, cudaStream_t st) {
  using V = typename C2<T>::type;
  const size_t smem = (size_t)2 * B * sizeof(V);
  cudaError_t e = cudaFuncSetAttribute(k_sft_to_xh<T, TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_sft_roots<T><<<(B + 255) / 256, 256, 0, st>>>(B, (V*)roots);
  const dim3 grid((unsigned)((B + kSftThreads * kSftOut - 1) / (kSftThreads * kSftOut)), (unsigned)n_sft);
  k_sft_to_xh<T, TIn><<<grid, kSftThreads, smem, st>>>((const TIn*)bins, (const V*)roots, B, f_het, t_start,
                                                       t_sft, 1.0 / (double)m_raw, (V*)xh);
  return cudaGetLastError();
}

}  // namespace

size_t sft_smem_bytes(int B, int precision) {
  return (size_t)2 * B * (precision == FSTAT_FP64 ? sizeof(double2) : sizeof(float2));
}

cudaError_t launch_sft_to_xh(int precision, int in_dtype, const void* bins, int64_t n_sft, int B, double f_het,
                             double t_start, double t_sft, int64_t m_raw, void* roots, void* xh,
                             cudaStream_t st) {
  const bool in64 = in_dtype == FSTAT_C128;
  if (precision == FSTAT_FP64)
    return in64 ? run_sft<double, double2>(bins, n_sft, B, f_het, t_start, t_sft, m_raw, roots, xh, st)
                : run_sft<double, float2>(bins, n_sft, B, f_het, t_start, t_sft, m_raw, roots, xh, st);
  return in64 ? run_sft<float, double2>(bins, n_sft, B, f_het, t_start, t_sft, m_raw, roots, xh, st)
              : run_sft<float, float2>(bins, n_sft, B, f_het, t_start, t_sft, m_raw, roots, xh, st);
}

}  // namespace fstat
