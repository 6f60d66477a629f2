// Step (ii) of Sec. 3 from short Fourier transforms (sft.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fstat {

// Shared memory of the transform kernel for a band of B bins.
size_t sft_smem_bytes(int B, int precision);
// x_h (n_sft * B samples, the plan's precision) from the band bins of
// n_sft SFTs; roots: device scratch of B 16-byte entries.
cudaError_t launch_sft_to_xh(int precision, int in_dtype, const void* bins, int64_t n_sft, int B, double f_het,
                             double t_start, double t_sft, int64_t m_raw, void* roots, void* xh,
                             cudaStream_t st);

}  // namespace fstat
