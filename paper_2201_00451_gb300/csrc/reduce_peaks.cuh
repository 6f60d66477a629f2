// Peaks reduction of dense 2F rows in device memory (reduce_peaks.cu).
#pragma once

#include "fstat_internal.cuh"

namespace fstat {

// n_rows rows of n_bins floats (n_bins a multiple of 4096); pk.tmpl is the
// index stored for row 0, pk.band_key the keys of row 0 (rows key_stride
// apart) or nullptr.
cudaError_t launch_reduce_peaks(const float* twoF, int64_t n_rows, int64_t n_bins, const PeakArgs& pk,
                                int64_t key_stride, cudaStream_t st);

}  // namespace fstat
