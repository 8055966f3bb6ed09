// Tables and the elementwise step of the spectral composition (Prop. 1, Eq. 4).
//
// U^T Lambda U = H^T (E Lambda E) H: with the unscaled cores H (the fused
// kernels) the diagonal is applied folded with the squared scales of Eq. 1,
// e_n[k] = 1/n (k = 0) or 2/n (k > 0) per axis; with scaled (orthonormal)
// transforms on both sides (the tensor-core route, and the forward -- scale
// -- inverse composition used for the other kernel families) it is Lambda
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

// One thread per four consecutive elements of an array row (w is a multiple
// of 4, every array start 16-byte aligned), grid-stride over the call.
__global__ void k_spectral_scale(float *out, const long long *out_off, long long count, int tiled, int tpr,
                                 long long ld, int h, int w, const float *lam)
{
    const int q = w / 4;                       // float4 per row
    const long long per = (long long)h * q;    // float4 per array
    const long long total = count * per;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long a = i / per;
        const int rem = (int)(i - a * per);
        const int r = rem / q, c4 = rem - r * q;
        float *row;
        if (tiled) {
            const long long br = a / tpr, bc = a - br * tpr;
            row = out + (br * h + r) * ld + bc * w;
        } else {
            row = (out_off ? out + out_off[a] : out + a * (long long)h * w) + (long long)r * w;
        }
        float4 *p = reinterpret_cast<float4 *>(row) + c4;
        const float4 d = __ldg(reinterpret_cast<const float4 *>(lam + (long long)r * w) + c4);
        float4 v = *p;
        v.x *= d.x; v.y *= d.y; v.z *= d.z; v.w *= d.w;
        *p = v;
    }
}

cudaError_t spectral_scale(const ExecGeom &g, int h, int w, const float *lam, cudaStream_t s)
{
    if (g.count <= 0) return cudaSuccess;
    if (w % 4) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long total = g.count * (long long)h * (w / 4);
    long long blocks = (total + 255) / 256;
    const long long cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    k_spectral_scale<<<(unsigned)blocks, 256, 0, s>>>(g.out, g.out_off, g.count, g.tiled, g.tiles_per_row, g.ld_out,
                                                      h, w, lam);
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
