// Tables of the spectral composition (Prop. 1, Eq. 4), and an array copy.
//
// U^T Lambda U = H^T (E Lambda E) H: with the unscaled cores H (the fused
// kernels) the diagonal is applied folded with the squared scales of Eq. 1,
// e_n[k] = 1/n (k = 0) or 2/n (k > 0) per axis; with scaled (orthonormal)
// transforms on both sides (the tensor-core routes, and the other kernel
// families, whose orthonormal forward multiplies its coefficients by the
// diagonal as it stores them before the orthonormal inverse) it is Lambda
// itself.  Both tables are computed in FP64 on the GPU and rounded once.
#include <cuda_runtime.h>

#include "bdct_internal.h"

namespace bdct {

__global__ void k_gen_spectral(const double *lam, float *plain, float *fold, int h, int w)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)h * w) return;
    const int k = (int)(idx / w), l = (int)(idx % w);
    const double eh = (k == 0 ? 1.0 : 2.0) / (double)h;
    const double ew = (l == 0 ? 1.0 : 2.0) / (double)w;
    const double v = lam[idx];
    plain[idx] = (float)v;
    fold[idx] = (float)(eh * v * ew);
}

cudaError_t spectral_gen_tables(const double *lam, float *plain, float *fold, int h, int w, cudaStream_t s)
{
    const long long n = (long long)h * w;
    k_gen_spectral<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(lam, plain, fold, h, w);
    return cudaGetLastError();
}

__global__ void k_copy_arrays(const float *src, float *out, const long long *out_off, long long count, int hw)
{
    const int q = hw / 4;
    const long long total = count * q;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long a = i / q;
        const int c4 = (int)(i - a * q);
        const float4 v = reinterpret_cast<const float4 *>(src + a * hw)[c4];
        reinterpret_cast<float4 *>(out_off ? out + out_off[a] : out + a * hw)[c4] = v;
    }
}

cudaError_t copy_arrays(const float *src, const ExecGeom &g, int h, int w, cudaStream_t s)
{
    if (g.count <= 0) return cudaSuccess;
    const int hw = h * w;
    if (hw % 4) return cudaErrorInvalidValue;
    if (!g.out_off) return cudaMemcpyAsync(g.out, src, (size_t)g.count * hw * sizeof(float), cudaMemcpyDeviceToDevice, s);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    long long blocks = (g.count * (hw / 4) + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    k_copy_arrays<<<(unsigned)blocks, 256, 0, s>>>(src, g.out, g.out_off, g.count, hw);
    return cudaGetLastError();
}

}  // namespace bdct
