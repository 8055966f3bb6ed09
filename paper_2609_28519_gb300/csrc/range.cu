// Numerical-range protection (the paper's Section 6 boundary diagnostics and
// its Section 8 future work: intermediates of the unnormalized cores can
// overflow although the orthonormal result is representable, and subnormal
// inputs lose relative accuracy).
//
// Every direction of the transform is linear, so T(X) = 2^e T(2^-e X)
// exactly in real arithmetic, and multiplying by a power of two is exact in
// floating point wherever the result stays normal.  With protection on, a
// call runs per chunk of arrays: (1) the largest magnitude of every array,
// (2) each array scaled by 2^-e with e its binary exponent (the largest
// magnitude moves into [1, 2): the cores' intermediates stay far from
// overflow and subnormal inputs become normal numbers), written to the output,
// (3) the transform in place on the output, (4) the output scaled back by 2^e.
// The cost is two extra reads and writes of the output and one extra read of
// the input.
#include <cuda_runtime.h>

#include "bdct_internal.h"

namespace bdct {

// Address of element (r, c) of array a of a call's geometry: contiguous,
// indexed through off, or tile a of an image with leading dimension ld.
__device__ __forceinline__ long long rp_index(long long a, int r, int c, int h, int w, const long long *off, int tiled,
                                              int tpr, long long ld)
{
    if (tiled) {
        const long long br = a / tpr, bc = a - br * tpr;
        return (br * h + r) * ld + bc * w + c;
    }
    return (off ? off[a] : a * (long long)h * w) + (long long)r * w + c;
}

// One block per (array, segment of up to 16384 elements): the largest
// magnitude, as the bits of a non-negative float (ordered like the values),
// merged into maxbits[a] with atomicMax.
__global__ void k_rp_max(const float *src, const long long *off, long long count, int tiled, int tpr, long long ld,
                         int h, int w, int segs, unsigned int *maxbits)
{
    const long long a = blockIdx.x / segs;
    const int seg = (int)(blockIdx.x - a * segs);
    const long long hw = (long long)h * w;
    const long long e0 = (long long)seg * 16384;
    long long e1 = e0 + 16384;
    if (e1 > hw) e1 = hw;
    unsigned int m = 0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int r = (int)(e / w), c = (int)(e - (long long)r * w);
        const float v = fabsf(src[rp_index(a, r, c, h, w, off, tiled, tpr, ld)]);
        const unsigned int b = __float_as_uint(v);
        // NaN compares above every finite value and infinity
        if (b > m) m = b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned int t = __shfl_xor_sync(0xffffffffu, m, o);
        if (t > m) m = t;
    }
    __shared__ unsigned int part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0u;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned int t = __shfl_xor_sync(0xffffffffu, m, o);
            if (t > m) m = t;
        }
        if (threadIdx.x == 0 && a < count) atomicMax(&maxbits[a], m);
    }
}

// Binary exponent of an array's largest magnitude (0 when it is zero,
// infinite or NaN: nothing to protect, nothing is scaled).
__device__ __forceinline__ int rp_exponent(unsigned int bits)
{
    if (bits == 0u || (bits >> 23) >= 255u) return 0;
    return ilogbf(__uint_as_float(bits));
}

// dst = src * 2^(sign * e_a) for every element, grid-stride; src and dst share
// the geometry's shape but may differ in base, offsets and leading dimension.
__global__ void k_rp_scale(const float *src, const long long *src_off, long long ld_src, float *dst,
                           const long long *dst_off, long long ld_dst, long long count, int tiled, int tpr, int h, int w,
                           const unsigned int *maxbits, int sign)
{
    const long long hw = (long long)h * w;
    const long long total = count * hw;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long a = i / hw;
        const long long e = i - a * hw;
        const int r = (int)(e / w), c = (int)(e - (long long)r * w);
        const int ex = rp_exponent(maxbits[a]);
        const float v = src[rp_index(a, r, c, h, w, src_off, tiled, tpr, ld_src)];
        dst[rp_index(a, r, c, h, w, dst_off, tiled, tpr, ld_dst)] = ldexpf(v, sign * ex);
    }
}

static cudaError_t grid_of(long long work, unsigned *blocks)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    long long b = (work + 255) / 256;
    if (b > (long long)sms * 16) b = (long long)sms * 16;
    if (b < 1) b = 1;
    *blocks = (unsigned)b;
    return cudaSuccess;
}

cudaError_t range_prescale(const ExecGeom &g, int h, int w, unsigned int *maxbits, cudaStream_t s)
{
    if (g.count <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(maxbits, 0, (size_t)g.count * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const long long hw = (long long)h * w;
    const int segs = (int)((hw + 16383) / 16384);
    const long long blocks = g.count * segs;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_rp_max<<<(unsigned)blocks, 256, 0, s>>>(g.in, g.in_off, g.count, g.tiled, g.tiles_per_row, g.ld_in, h, w, segs,
                                             maxbits);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    unsigned nb = 0;
    e = grid_of(g.count * hw, &nb);
    if (e != cudaSuccess) return e;
    k_rp_scale<<<nb, 256, 0, s>>>(g.in, g.in_off, g.ld_in, g.out, g.out_off, g.ld_out, g.count, g.tiled,
                                  g.tiles_per_row, h, w, maxbits, -1);
    return cudaGetLastError();
}

cudaError_t range_postscale(const ExecGeom &g, int h, int w, const unsigned int *maxbits, cudaStream_t s)
{
    if (g.count <= 0) return cudaSuccess;
    unsigned nb = 0;
    cudaError_t e = grid_of(g.count * (long long)h * w, &nb);
    if (e != cudaSuccess) return e;
    k_rp_scale<<<nb, 256, 0, s>>>(g.out, g.out_off, g.ld_out, g.out, g.out_off, g.ld_out, g.count, g.tiled,
                                  g.tiles_per_row, h, w, maxbits, 1);
    return cudaGetLastError();
}

}  // namespace bdct
