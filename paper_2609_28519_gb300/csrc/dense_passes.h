// Entry points of the dense passes beyond those in bdct_internal.h.
#pragma once

#include <cuda_runtime.h>

namespace bdct {

// dense_pass_cols with every output element (k, l) of an array multiplied by
// lam[k * w + l] (or dense_pass_cols itself for lam null): the forward's
// second pass times the diagonal, the first half of the spectral composition
// of Prop. 1 (Eq. 4) on the dense route.
cudaError_t dense_pass_cols_lam(const float *in, float *out, const float *op_h, int h, int w, long long count,
                                const float *lam, cudaStream_t stream);

}  // namespace bdct
