// Register-resident 1D DCT/FFT cores shared by the FP32 kernels.
//
// Exact factorizations of the unscaled kernels of Eq. 1 (no approximated
// coefficient):
//  * DCT-II of length N splits into a DCT-II of length N/2 on the sums
//    x_j + x_{N-1-j} (even outputs) and a DCT-IV of length N/2 on the
//    differences (odd outputs);
//  * DCT-III (the adjoint) reverses this: DCT-III of the even inputs, DCT-IV
//    of the odd inputs, then a sum/difference butterfly;
//  * DCT-IV of length M > 4 is a pre-twiddle of M/2 complex points, a
//    length-M/2 complex FFT (radix-2, decimation in time) and a post-twiddle;
//    M <= 4 is a direct matrix product.
// Every compile-time twiddle comes from the FP32 table c_cos[r] = cos(pi r /
// 8192), built on the GPU in FP64; each translation unit that includes this
// header owns a copy and fills it through init_cos_table().
#pragma once

#include <cuda_runtime.h>

#include "bdct_internal.h"

namespace bdct {

static __constant__ float c_cos[4097];  // cos(pi r / 8192), r = 0..4096 (one copy per translation unit)

// ------------------------------------------------------------ twiddles
// cos(pi m / d) for d a power of two dividing 8192; m may be negative.
__device__ __forceinline__ float cospi_md(int m, int d)
{
    int r = (m * (8192 / d)) & 16383;
    if (r > 8192) r = 16384 - r;
    if (r == 0) return 1.0f;
    if (r == 8192) return -1.0f;
    if (r == 4096) return 0.0f;
    return (r > 4096) ? -c_cos[8192 - r] : c_cos[r];
}
// sin(pi m / d) = cos(pi (d/2 - m) / d)
__device__ __forceinline__ float sinpi_md(int m, int d) { return cospi_md(d / 2 - m, d); }

// (ar + i ai) * exp(-i pi m / d), with the trivial angles resolved at compile time.
__device__ __forceinline__ void rot(float ar, float ai, int m, int d, float &rr, float &ri)
{
    int r = (m * (8192 / d)) & 16383;
    if (r == 0) { rr = ar; ri = ai; return; }
    if (r == 8192) { rr = -ar; ri = -ai; return; }
    if (r == 4096) { rr = ai; ri = -ar; return; }
    if (r == 12288) { rr = -ai; ri = ar; return; }
    float c = cospi_md(m, d), s = sinpi_md(m, d);
    rr = fmaf(ar, c, ai * s);
    ri = fmaf(ai, c, -(ar * s));
}

// ------------------------------------------------------------ 1D cores
// Forward complex DFT X_k = sum_j x_j exp(-2 pi i j k / L), radix-2 DIT.
// Twiddles for lengths with a factor 3: c_cos3[r] = cos(pi r / 1536),
// r = 0..768 (one copy per translation unit, filled by init_cos_table3).
static __constant__ float c_cos3[769];

// cos(pi m / d) for d dividing 1536 * 2 (lengths 3 * 2^k <= 3072).
__device__ __forceinline__ float cospi3_md(int m, int d)
{
    int r = (m * (1536 / d)) % 3072;
    if (r < 0) r += 3072;
    if (r > 1536) r = 3072 - r;
    if (r == 0) return 1.0f;
    if (r == 1536) return -1.0f;
    if (r == 768) return 0.0f;
    return (r > 768) ? -c_cos3[1536 - r] : c_cos3[r];
}
__device__ __forceinline__ float sinpi3_md(int m, int d) { return cospi3_md(d / 2 - m, d); }

// (ar + i ai) * exp(-2 pi i k / L) for L = 3 * 2^j.
__device__ __forceinline__ void rot3(float ar, float ai, int k, int L, float &rr, float &ri)
{
    if (k % L == 0) { rr = ar; ri = ai; return; }
    const float c = cospi3_md(2 * k, L), s = sinpi3_md(2 * k, L);
    rr = fmaf(ar, c, ai * s);
    ri = fmaf(ai, c, -(ar * s));
}

template <int L>
struct FFT {
    static __device__ __forceinline__ void run(float (&re)[L], float (&im)[L])
    {
        if constexpr (L % 3 == 0) {
            // radix-3 decimation in time: three interleaved FFTs of L/3, then a
            // 3-point DFT of (E0_k, w^k E1_k, w^2k E2_k), w = exp(-2 pi i / L)
            constexpr int M = L / 3;
            float r0[M], i0[M], r1[M], i1[M], r2[M], i2[M];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                r0[j] = re[3 * j]; i0[j] = im[3 * j];
                r1[j] = re[3 * j + 1]; i1[j] = im[3 * j + 1];
                r2[j] = re[3 * j + 2]; i2[j] = im[3 * j + 2];
            }
            FFT<M>::run(r0, i0);
            FFT<M>::run(r1, i1);
            FFT<M>::run(r2, i2);
            const float h = cospi3_md(256, 1536);  // cos(pi / 6) = sqrt(3) / 2
#pragma unroll
            for (int k = 0; k < M; ++k) {
                float br, bi, cr, ci;
                rot3(r1[k], i1[k], k, L, br, bi);
                rot3(r2[k], i2[k], 2 * k, L, cr, ci);
                const float tr = br + cr, ti = bi + ci;      // b + c
                const float dr = br - cr, di = bi - ci;      // b - c
                const float mr = r0[k] - 0.5f * tr, mi = i0[k] - 0.5f * ti;
                // -i sqrt(3)/2 (b - c)
                const float sr = h * di, si = -h * dr;
                re[k] = r0[k] + tr; im[k] = i0[k] + ti;
                re[k + M] = mr + sr; im[k + M] = mi + si;
                re[k + 2 * M] = mr - sr; im[k + 2 * M] = mi - si;
            }
        } else {
            radix2(re, im);
        }
    }

    // radix-2 decimation in time: two interleaved FFTs of L/2, then butterflies
    static __device__ __forceinline__ void radix2(float (&re)[L], float (&im)[L])
    {
        float er[L / 2], ei[L / 2], orr[L / 2], oi[L / 2];
#pragma unroll
        for (int j = 0; j < L / 2; ++j) {
            er[j] = re[2 * j]; ei[j] = im[2 * j];
            orr[j] = re[2 * j + 1]; oi[j] = im[2 * j + 1];
        }
        FFT<L / 2>::run(er, ei);
        FFT<L / 2>::run(orr, oi);
#pragma unroll
        for (int k = 0; k < L / 2; ++k) {
            float tr, ti;
            rot(orr[k], oi[k], 2 * k, L, tr, ti);  // exp(-2 pi i k / L), L a power of two
            re[k] = er[k] + tr; im[k] = ei[k] + ti;
            re[k + L / 2] = er[k] - tr; im[k + L / 2] = ei[k] - ti;
        }
    }
};
template <>
struct FFT<1> {
    static __device__ __forceinline__ void run(float (&)[1], float (&)[1]) {}
};

// DCT-IV: z_k = sum_j v_j cos(pi (2j+1)(2k+1) / (4M)).  Symmetric matrix.
template <int M>
struct DCT4 {
    static __device__ __forceinline__ void run(const float (&v)[M], float (&z)[M])
    {
        if constexpr (M <= 4) {
#pragma unroll
            for (int k = 0; k < M; ++k) {
                float acc = v[0] * cospi_md(2 * k + 1, 4 * M);
#pragma unroll
                for (int j = 1; j < M; ++j) acc = fmaf(v[j], cospi_md((2 * j + 1) * (2 * k + 1), 4 * M), acc);
                z[k] = acc;
            }
        } else {
            // u_j = (v_{2j} + i v_{M-1-2j}) exp(-i pi (4j+1) / (4M))
            float ur[M / 2], ui[M / 2];
#pragma unroll
            for (int j = 0; j < M / 2; ++j) rot(v[2 * j], v[M - 1 - 2 * j], 4 * j + 1, 4 * M, ur[j], ui[j]);
            FFT<M / 2>::run(ur, ui);
            // W_k = U_k exp(-i pi k / M); z_{2k} = Re W_k, z_{M-1-2k} = -Im W_k
#pragma unroll
            for (int k = 0; k < M / 2; ++k) {
                float wr, wi;
                rot(ur[k], ui[k], k, M, wr, wi);
                z[2 * k] = wr;
                z[M - 1 - 2 * k] = -wi;
            }
        }
    }
};

// Unscaled DCT-II: y_k = sum_j x_j cos(pi (2j+1) k / (2N)).
template <int N>
struct DCT2 {
    static __device__ __forceinline__ void run(const float (&x)[N], float (&y)[N])
    {
        float u[N / 2], v[N / 2], ye[N / 2], yo[N / 2];
#pragma unroll
        for (int j = 0; j < N / 2; ++j) {
            u[j] = x[j] + x[N - 1 - j];
            v[j] = x[j] - x[N - 1 - j];
        }
        DCT2<N / 2>::run(u, ye);
        DCT4<N / 2>::run(v, yo);
#pragma unroll
        for (int m = 0; m < N / 2; ++m) { y[2 * m] = ye[m]; y[2 * m + 1] = yo[m]; }
    }
};
template <>
struct DCT2<1> {
    static __device__ __forceinline__ void run(const float (&x)[1], float (&y)[1]) { y[0] = x[0]; }
};

// Unscaled DCT-III (transpose of DCT2): x_j = sum_k y_k cos(pi (2j+1) k / (2N)).
template <int N>
struct DCT3 {
    static __device__ __forceinline__ void run(const float (&y)[N], float (&x)[N])
    {
        float ye[N / 2], yo[N / 2], a[N / 2], b[N / 2];
#pragma unroll
        for (int m = 0; m < N / 2; ++m) { ye[m] = y[2 * m]; yo[m] = y[2 * m + 1]; }
        DCT3<N / 2>::run(ye, a);
        DCT4<N / 2>::run(yo, b);
#pragma unroll
        for (int j = 0; j < N / 2; ++j) {
            x[j] = a[j] + b[j];
            x[N - 1 - j] = a[j] - b[j];
        }
    }
};
template <>
struct DCT3<1> {
    static __device__ __forceinline__ void run(const float (&y)[1], float (&x)[1]) { x[0] = y[0]; }
};

template <int N>
__device__ __forceinline__ void scale_line(float (&x)[N], AxisScale s)
{
    x[0] *= s.s0;
#pragma unroll
    for (int k = 1; k < N; ++k) x[k] *= s.s1;
}

// One direction of the 2D transform along one axis of a line held in registers.
template <int N, int DIR>
__device__ __forceinline__ void line_op(float (&x)[N], AxisScale s)
{
    float y[N];
    if constexpr (DIR == DIR_FWD) {
        DCT2<N>::run(x, y);
        scale_line<N>(y, s);
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = y[k];
    } else if constexpr (DIR == DIR_INV) {
        scale_line<N>(x, s);
        DCT3<N>::run(x, y);
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = y[k];
    } else {
        DCT2<N>::run(x, y);
        scale_line<N>(y, s);
        DCT3<N>::run(y, x);
    }
}


// Fill this translation unit's constant table from a device buffer holding
// cos(pi r / 8192), r = 0..4096.
static inline cudaError_t init_cos_table(const float *d_table)
{
    return cudaMemcpyToSymbol(c_cos, d_table, 4097 * sizeof(float), 0, cudaMemcpyDeviceToDevice);
}

// Same for the radix-3 table: a device buffer holding cos(pi r / 1536), r = 0..768.
static inline cudaError_t init_cos_table3(const float *d_table)
{
    return cudaMemcpyToSymbol(c_cos3, d_table, 769 * sizeof(float), 0, cudaMemcpyDeviceToDevice);
}

}  // namespace bdct
