// Entry points of the line engine beyond lines_pass (fp32_lines.cu).
#pragma once

#include <cuda_runtime.h>

#include "bdct_internal.h"

namespace bdct {

// lines_pass with every output element (k, r) of an array (k < n the
// transformed index, r < rows the line) multiplied by lam[k * rows + r] as
// it is stored, or lines_pass itself for lam null: the second pass of a
// forward transform times the diagonal, the first half of the spectral
// composition of Prop. 1 (Eq. 4) on the line engine.  lam is 16-byte
// aligned, rows a multiple of 4.
cudaError_t lines_pass_lam(const float *src, float *dst, int rows, int n, long long count, Dir dir, AxisScale sc,
                           const float2 *tw, unsigned int *status, cudaStream_t stream, const long long *src_off,
                           const long long *dst_off, bool reverse, const float *lam);

}  // namespace bdct
