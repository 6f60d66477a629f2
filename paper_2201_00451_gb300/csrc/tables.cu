// Twiddle tables for the FFT passes: roots of unity exp(-2 pi i m / M),
// evaluated in FP64 (sincospi) and stored in the path's precision.
//
// Layout of one table block for n_fft = N1 * N2 = 2^(l1 + l2):
//   [ tw_A : N2 entries, M = N2 ]   Stockham twiddles of pass A
//   [ tw_B : N1 entries, M = N1 ]   Stockham twiddles of pass B
// (the four-step twiddles W_N^{n1 k2} are computed in pass A itself)
#include "fstat_internal.cuh"

namespace fstat {
namespace {

template <typename TW>
__global__ void k_roots(TW* out, int count, int log2m) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double x = -2.0 * (double)i / (double)(1 << log2m);
  double s, c;
  sincospi(x, &s, &c);
  TW w;
  w.x = c;
  w.y = s;
  out[i] = w;
}

template <typename TW>
void roots(TW* out, int log2m, cudaStream_t st) {
  int count = 1 << log2m;
  k_roots<TW><<<(count + 255) / 256, 256, 0, st>>>(out, count, log2m);
}

}  // namespace

int device_sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (!cached[dev]) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    cached[dev] = sms;
  }
  return cached[dev];
}

TwiddleTables twiddle_layout(int precision, int log2n1, int log2n2, void* base) {
  TwiddleTables t{};
  const size_t eb = precision == FSTAT_FP64 ? 16 : 8;
  char* p = (char*)base;
  t.a = p; p += eb * ((size_t)1 << log2n2);
  t.b = p; p += eb * ((size_t)1 << log2n1);
  t.bytes = (size_t)(p - (char*)base);
  return t;
}

cudaError_t build_twiddles(int precision, int log2n1, int log2n2, void* base, cudaStream_t st) {
  TwiddleTables t = twiddle_layout(precision, log2n1, log2n2, base);
  if (precision == FSTAT_FP64) {
    roots((double2*)t.a, log2n2, st);
    roots((double2*)t.b, log2n1, st);
  } else {
    roots((float2*)t.a, log2n2, st);
    roots((float2*)t.b, log2n1, st);
  }
  return cudaGetLastError();
}

}  // namespace fstat
