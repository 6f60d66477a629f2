// fstat_twoF_noalloc: one template's 2F from a caller-resampled series,
// without any device allocation.
//
// Some callers cannot call cudaMalloc: a plug-in running inside a host
// application whose memory pool already owns the device memory and forbids
// outside allocations, and a low-latency pipeline that must not allocate
// after start-up because cudaMalloc can synchronise the device and has no
// latency bound.  This entry point keeps its working memory in file-scope
// __device__ arrays of fixed size (8.1 MB).  With CUDA's lazy module loading
// (the default since CUDA 12.2) the arrays are reserved on a device when
// this file's module is first used there, i.e. by the first call on that
// device; from then on the device holds them until the process exits.  A
// caller whose pool takes the rest of the device memory should make that
// first call at start-up, before the pool claims the memory.
//
// It runs the same FFT pass kernels as fstat_compute (spindown phase +
// column FFTs, then row FFTs + eq. Fstat); only the scratch memory differs.

#include <math.h>

#include <atomic>
#include <mutex>

#include "fstat_internal.cuh"

namespace fstat {
namespace {

constexpr int kNoallocMaxLog2 = 18;  // n_fft <= 2^18
constexpr int64_t kNoallocMaxFft = int64_t(1) << kNoallocMaxLog2;
constexpr int64_t kNoallocGElems = kNoallocMaxFft + (int64_t(1) << kMaxLog2);

// Scratch: column-major copy of the input pairs, the FFT intermediate, the
// twiddle tables and the per-call constants: 4.06 MB + 4 MB + 16 KB per device.
static __device__ __align__(256) float4 g_scratch_G[kNoallocGElems];
static __device__ __align__(256) float4 g_scratch_Z[kNoallocMaxFft];
static __device__ __align__(256) float2 g_scratch_tw[4 * (1 << (kNoallocMaxLog2 / 2))];
static __device__ __align__(256) SkyConst g_scratch_sky;
static __device__ __align__(256) TmplCoef g_scratch_coef;

constexpr int kMaxDevices = 64;
struct DevPtrs {
  float4* G;
  float4* Z;
  float2* tw;
  SkyConst* sky;
  TmplCoef* coef;
};
std::mutex g_setup_mutex;
DevPtrs g_ptrs[kMaxDevices];
std::atomic<bool> g_ready[kMaxDevices];

// Device addresses of the scratch arrays on the current device (host code
// sees only host-side stand-ins for the symbols).
int device_ptrs(DevPtrs* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FSTAT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return FSTAT_ERR_UNSUPPORTED;
  if (!g_ready[dev].load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_ready[dev].load(std::memory_order_relaxed)) {
      DevPtrs p{};
      if (cudaGetSymbolAddress((void**)&p.G, g_scratch_G) != cudaSuccess) return FSTAT_ERR_CUDA;
      if (cudaGetSymbolAddress((void**)&p.Z, g_scratch_Z) != cudaSuccess) return FSTAT_ERR_CUDA;
      if (cudaGetSymbolAddress((void**)&p.tw, g_scratch_tw) != cudaSuccess) return FSTAT_ERR_CUDA;
      if (cudaGetSymbolAddress((void**)&p.sky, g_scratch_sky) != cudaSuccess) return FSTAT_ERR_CUDA;
      if (cudaGetSymbolAddress((void**)&p.coef, g_scratch_coef) != cudaSuccess) return FSTAT_ERR_CUDA;
      g_ptrs[dev] = p;
      g_ready[dev].store(true, std::memory_order_release);
    }
  }
  *out = g_ptrs[dev];
  return FSTAT_OK;
}

// Per-call constants: 2F weights from A, B, C and the spindown polynomial
// in s = j - J for tau_j = tau0 + j dt = (j - j_ref) dt, j_ref = -tau0 / dt.
__global__ void k_noalloc_setup(double A, double B, double C, double tau0, double dt, int64_t n,
                                double f1dot, double f2dot) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double D = A * B - C * C;
  g_scratch_sky.A = A;
  g_scratch_sky.B = B;
  g_scratch_sky.C = C;
  g_scratch_sky.D = D;
  g_scratch_sky.kA = 2.0 * A / D;
  g_scratch_sky.kB = 2.0 * B / D;
  g_scratch_sky.kC = 4.0 * C / D;
  g_scratch_sky.kAf = (float)g_scratch_sky.kA;
  g_scratch_sky.kBf = (float)g_scratch_sky.kB;
  g_scratch_sky.kCf = (float)g_scratch_sky.kC;
  g_scratch_coef = spin_coef(-tau0 / dt, n, dt, f1dot, f2dot);
}

// natural order j -> column-major [(j mod n1) * lc + j / n1]
__global__ void k_noalloc_columns(const float4* __restrict__ g, int64_t n, int n1, int64_t lc,
                                  float4* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[(j % n1) * lc + j / n1] = g[j];
}

}  // namespace
}  // namespace fstat

using namespace fstat;

extern "C" int fstat_twoF_noalloc(const void* g_pairs, int64_t n_samples, int64_t n_fft, double dt,
                                  double tau0, double A, double B, double C, double f1dot,
                                  double f2dot, float* twoF, void* stream) {
  if (!g_pairs || !twoF || n_samples < 1 || !(dt > 0.0) || !isfinite(tau0) || !isfinite(f1dot) ||
      !isfinite(f2dot) || !isfinite(A) || !isfinite(B) || !isfinite(C))
    return FSTAT_ERR_INVALID_ARG;
  if (n_fft <= 0 || (n_fft & (n_fft - 1))) return FSTAT_ERR_INVALID_ARG;
  int log2n = 0;
  while ((int64_t(1) << log2n) < n_fft) ++log2n;
  if (n_fft > kNoallocMaxFft || log2n < 2 * kMinLog2) return FSTAT_ERR_UNSUPPORTED;
  if (n_samples > n_fft) return FSTAT_ERR_INVALID_ARG;
  double D = A * B - C * C;
  if (!(D > 1e-12 * A * B) || !(A > 0.0) || !(B > 0.0)) return FSTAT_ERR_DEGENERATE;
  // spindown phase excursion over the data within what the phase evaluation
  // reduces exactly (this also bounds |tau0|)
  const double tmax = fmax(fabs(tau0), fabs(tau0 + (double)(n_samples - 1) * dt)) + dt;
  if (!spin_in_range(tmax, f1dot, f2dot)) return FSTAT_ERR_UNSUPPORTED;

  DevPtrs p;
  int rc = device_ptrs(&p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int log2n1 = log2n / 2, log2n2 = log2n - log2n1;
  const int n1 = 1 << log2n1, n2 = 1 << log2n2;
  const int64_t lc = (n_samples + n1 - 1) / n1;

  k_noalloc_setup<<<1, 32, 0, st>>>(A, B, C, tau0, dt, n_samples, f1dot, f2dot);
  int blocks = (int)((n_samples + 255) / 256);
  if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
  k_noalloc_columns<<<blocks, 256, 0, st>>>((const float4*)g_pairs, n_samples, n1, lc, p.G);
  if (cudaGetLastError() != cudaSuccess) return FSTAT_ERR_CUDA;
  cudaError_t e = build_twiddles(FSTAT_MIXED, log2n1, log2n2, p.tw, st);
  if (e != cudaSuccess) return FSTAT_ERR_CUDA;
  TwiddleTables tt = twiddle_layout(FSTAT_MIXED, log2n1, log2n2, p.tw);
  e = launch_pass_a_f32(log2n2, 0, 0, p.G, lc, n_samples, n1, tt.a, p.coef, p.Z, st);
  if (e != cudaSuccess) return FSTAT_ERR_CUDA;
  e = launch_pass_b_f32(log2n1, 0, 0, p.Z, n2, tt.b, p.sky, twoF, st);
  if (e != cudaSuccess) return FSTAT_ERR_CUDA;
  return FSTAT_OK;
}
