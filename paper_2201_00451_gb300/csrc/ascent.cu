// Gradient-ascent steps of fstat_refine (see ascent.cuh): one thread per
// candidate, FP64 parameters.  Refinement is an extension of the method:
// grid candidates are followed up off the grid by ascending eq. (Fstat),
// evaluated with the demodulation sums of Sec. 2, along the gradient that
// fstat_grad's adjoint kernels return.
#include "ascent.cuh"

namespace fstat {
namespace {

struct Scales {
  double s[4];
};

__global__ void k_ascent_init(AscentState s, double step0, float* __restrict__ hist_row) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  s.eta[i] = step0;
  if (hist_row) hist_row[i] = s.cur[i];
}

// Every product and sum rounded on its own (no contraction), so the step is
// the same double as the textbook expression evaluated left to right.
__device__ __forceinline__ double move(double th, double step, double sg, double sc) {
  return __dadd_rn(th, __dmul_rn(__dmul_rn(step, sg), sc));
}

__global__ void k_ascent_trial(AscentState s, Scales sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const fstat_candidate th = s.theta[i];
  double sg[4], nrm2 = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    sg[j] = __dmul_rn((double)s.g[4 * i + j], sc.s[j]);
    nrm2 = __dadd_rn(nrm2, __dmul_rn(sg[j], sg[j]));
  }
  const double step = s.eta[i] / fmax(sqrt(nrm2), 1e-300);
  fstat_candidate tr = th;
  tr.f = move(th.f, step, sg[0], sc.s[0]);
  tr.f1dot = move(th.f1dot, step, sg[1], sc.s[1]);
  tr.alpha = move(th.alpha, step, sg[2], sc.s[2]);
  tr.delta = move(th.delta, step, sg[3], sc.s[3]);
  s.trial[i] = tr;
}

__global__ void k_ascent_accept(AscentState s, float* __restrict__ hist_row) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const float v = s.val[i];
  // a NaN trial value is never taken
  if (v > s.cur[i]) {
    s.theta[i] = s.trial[i];
    s.cur[i] = v;
#pragma unroll
    for (int j = 0; j < 4; ++j) s.g[4 * i + j] = s.gt[4 * i + j];
    s.eta[i] *= 1.25;
  } else {
    s.eta[i] *= 0.5;
  }
  if (hist_row) hist_row[i] = s.cur[i];
}

int blocks(int n) { return (n + 127) / 128; }

}  // namespace

cudaError_t launch_ascent_init(const AscentState& s, double step0, float* hist_row, cudaStream_t st) {
  if (s.n <= 0) return cudaSuccess;
  k_ascent_init<<<blocks(s.n), 128, 0, st>>>(s, step0, hist_row);
  return cudaGetLastError();
}

cudaError_t launch_ascent_trial(const AscentState& s, const double* scales, cudaStream_t st) {
  if (s.n <= 0) return cudaSuccess;
  Scales sc;
  for (int j = 0; j < 4; ++j) sc.s[j] = scales[j];
  k_ascent_trial<<<blocks(s.n), 128, 0, st>>>(s, sc);
  return cudaGetLastError();
}

cudaError_t launch_ascent_accept(const AscentState& s, float* hist_row, cudaStream_t st) {
  if (s.n <= 0) return cudaSuccess;
  k_ascent_accept<<<blocks(s.n), 128, 0, st>>>(s, hist_row);
  return cudaGetLastError();
}

}  // namespace fstat
