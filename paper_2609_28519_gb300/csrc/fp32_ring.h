// Entry points of the ring kernels beyond ring_launch (fp32_ring.cu).
#pragma once

#include <cuda_runtime.h>

#include "bdct_internal.h"

namespace bdct {

// Forward transform of 64 x 128, 128 x 64 or 128 x 128 arrays with every
// coefficient multiplied by g.lam (rows x cols, row k = frequency along h)
// as it is stored: the first half of the spectral composition of Prop. 1
// (Eq. 4) for the ring shapes whose direction is not fused whole; the
// orthonormal inverse completes it.
cudaError_t ring_forward_lam(int rows, int cols, const DirScales &sc, const ExecGeom &g, unsigned int *status,
                             cudaStream_t stream);

}  // namespace bdct
