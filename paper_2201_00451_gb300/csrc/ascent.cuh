// Gradient ascent on 2F over refinement candidates, on the device (the loop
// of fstat_refine): trial points and the accept / reject rule between the
// adjoint evaluations, so that the loop needs no host round trip.
#pragma once

#include "fstat_internal.cuh"

namespace fstat {

// Ascent state of n candidates, all DEVICE arrays: theta (the accepted
// candidates), trial, cur / val (2F at theta / trial), g / gt (d2F/dtheta at
// theta / trial, 4 floats each), eta (step length in scaled units).
struct AscentState {
  fstat_candidate* theta;
  fstat_candidate* trial;
  float* cur;
  float* val;
  float* g;
  float* gt;
  double* eta;
  int n;
};

// eta = step0, hist row 0 = cur (after the first evaluation at theta)
cudaError_t launch_ascent_init(const AscentState& s, double step0, float* hist_row, cudaStream_t st);
// trial = theta + eta / |g * sc| (g * sc) * sc, per candidate (sc: the
// natural spacings of f, f1dot, alpha, delta)
cudaError_t launch_ascent_trial(const AscentState& s, const double* sc, cudaStream_t st);
// val > cur: take the trial (theta, cur, g) and eta *= 1.25; else eta *= 0.5;
// hist row = cur
cudaError_t launch_ascent_accept(const AscentState& s, float* hist_row, cudaStream_t st);

}  // namespace fstat
