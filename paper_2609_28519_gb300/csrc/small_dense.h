// On-chip dense route for small arrays (small_dense.cu).
#pragma once

#include <cuda_runtime.h>

#include "bdct_internal.h"

namespace bdct {

// Both sides at most 64 and the width a multiple of 4.
bool small_dense_supported(int h, int w);

// `npass` (2 to 4) passes over the arrays of `g`, in shared memory: pass q
// applies the n x n row-major operator op[q] (y = M x, scales folded in)
// along w (axis[q] == 0, every row) or along h (axis[q] == 1, every column);
// with `lam`, the h x w diagonal multiplies the result of the second pass.
// The arrays are a contiguous batch, indexed arrays (element offsets) or the
// tiles of an image (leading dimensions multiples of 4).  In place is
// allowed.
cudaError_t small_dense_run(int h, int w, int npass, const int *axis, const float *const *op, const float *lam,
                            const ExecGeom &g, cudaStream_t stream);

}  // namespace bdct
