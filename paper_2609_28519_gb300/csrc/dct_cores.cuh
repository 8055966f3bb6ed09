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

// ------------------------------------------------------------ value types
// Every core runs on one line (V = float) or on two lines at once (V =
// float2): the packed FP32 instructions of sm_100-family GPUs apply one
// add, multiply or fused multiply-add to both halves of a register pair, so
// two lines cost the instructions of one.  Each packed operation rounds each
// half exactly as the scalar operation does.
template <typename V>
struct VOps;
template <>
struct VOps<float> {
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
    static __device__ __forceinline__ float mul(float a, float c) { return a * c; }
    static __device__ __forceinline__ float fma(float a, float c, float b) { return fmaf(a, c, b); }
    static __device__ __forceinline__ float neg(float a) { return -a; }
};
template <>
struct VOps<float2> {
    static __device__ __forceinline__ float2 dup(float c) { return make_float2(c, c); }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    // a - b as a + (-1) b: one rounding, the value of the subtraction
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, dup(-1.0f), a); }
    static __device__ __forceinline__ float2 mul(float2 a, float c) { return __fmul2_rn(a, dup(c)); }
    static __device__ __forceinline__ float2 fma(float2 a, float c, float2 b) { return __ffma2_rn(a, dup(c), b); }
    static __device__ __forceinline__ float2 neg(float2 a) { return __fmul2_rn(a, dup(-1.0f)); }
};
template <typename V>
inline constexpr bool kPacked = sizeof(V) == 8;

// (ar + i ai) * exp(-i pi m / d), with the trivial angles resolved at compile time.
template <typename V>
__device__ __forceinline__ void rot(V ar, V ai, int m, int d, V &rr, V &ri)
{
    using O = VOps<V>;
    int r = (m * (8192 / d)) & 16383;
    if (r == 0) { rr = ar; ri = ai; return; }
    if (r == 8192) { rr = O::neg(ar); ri = O::neg(ai); return; }
    if (r == 4096) { rr = ai; ri = O::neg(ar); return; }
    if (r == 12288) { rr = O::neg(ai); ri = ar; return; }
    float c = cospi_md(m, d), s = sinpi_md(m, d);
    rr = O::fma(ar, c, O::mul(ai, s));
    ri = O::fma(ai, c, O::mul(ar, -s));
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
template <typename V>
__device__ __forceinline__ void rot3(V ar, V ai, int k, int L, V &rr, V &ri)
{
    using O = VOps<V>;
    if (k % L == 0) { rr = ar; ri = ai; return; }
    const float c = cospi3_md(2 * k, L), s = sinpi3_md(2 * k, L);
    rr = O::fma(ar, c, O::mul(ai, s));
    ri = O::fma(ai, c, O::mul(ar, -s));
}

template <int L, typename V = float>
struct FFT {
    using O = VOps<V>;
    static __device__ __forceinline__ void run(V (&re)[L], V (&im)[L])
    {
        if constexpr (L % 3 == 0) {
            // radix-3 decimation in time: three interleaved FFTs of L/3, then a
            // 3-point DFT of (E0_k, w^k E1_k, w^2k E2_k), w = exp(-2 pi i / L)
            constexpr int M = L / 3;
            V r0[M], i0[M], r1[M], i1[M], r2[M], i2[M];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                r0[j] = re[3 * j]; i0[j] = im[3 * j];
                r1[j] = re[3 * j + 1]; i1[j] = im[3 * j + 1];
                r2[j] = re[3 * j + 2]; i2[j] = im[3 * j + 2];
            }
            FFT<M, V>::run(r0, i0);
            FFT<M, V>::run(r1, i1);
            FFT<M, V>::run(r2, i2);
            const float h = cospi3_md(256, 1536);  // cos(pi / 6) = sqrt(3) / 2
#pragma unroll
            for (int k = 0; k < M; ++k) {
                V br, bi, cr, ci;
                rot3(r1[k], i1[k], k, L, br, bi);
                rot3(r2[k], i2[k], 2 * k, L, cr, ci);
                const V tr = O::add(br, cr), ti = O::add(bi, ci);  // b + c
                const V dr = O::sub(br, cr), di = O::sub(bi, ci);  // b - c
                const V mr = O::fma(tr, -0.5f, r0[k]), mi = O::fma(ti, -0.5f, i0[k]);
                // -i sqrt(3)/2 (b - c)
                const V sr = O::mul(di, h), si = O::mul(dr, -h);
                re[k] = O::add(r0[k], tr); im[k] = O::add(i0[k], ti);
                re[k + M] = O::add(mr, sr); im[k + M] = O::add(mi, si);
                re[k + 2 * M] = O::sub(mr, sr); im[k + 2 * M] = O::sub(mi, si);
            }
        } else {
            radix2(re, im);
        }
    }

    // radix-2 decimation in time: two interleaved FFTs of L/2, then butterflies
    static __device__ __forceinline__ void radix2(V (&re)[L], V (&im)[L])
    {
        V er[L / 2], ei[L / 2], orr[L / 2], oi[L / 2];
#pragma unroll
        for (int j = 0; j < L / 2; ++j) {
            er[j] = re[2 * j]; ei[j] = im[2 * j];
            orr[j] = re[2 * j + 1]; oi[j] = im[2 * j + 1];
        }
        FFT<L / 2, V>::run(er, ei);
        FFT<L / 2, V>::run(orr, oi);
#pragma unroll
        for (int k = 0; k < L / 2; ++k) {
            V tr, ti;
            rot(orr[k], oi[k], 2 * k, L, tr, ti);  // exp(-2 pi i k / L), L a power of two
            re[k] = O::add(er[k], tr); im[k] = O::add(ei[k], ti);
            re[k + L / 2] = O::sub(er[k], tr); im[k + L / 2] = O::sub(ei[k], ti);
        }
    }
};
template <typename V>
struct FFT<1, V> {
    static __device__ __forceinline__ void run(V (&)[1], V (&)[1]) {}
};

// DCT-IV: z_k = sum_j v_j cos(pi (2j+1)(2k+1) / (4M)).  Symmetric matrix.
template <int M, typename V = float>
struct DCT4 {
    using O = VOps<V>;
    static __device__ __forceinline__ void run(const V (&v)[M], V (&z)[M])
    {
        if constexpr (M <= 4) {
#pragma unroll
            for (int k = 0; k < M; ++k) {
                V acc = O::mul(v[0], cospi_md(2 * k + 1, 4 * M));
#pragma unroll
                for (int j = 1; j < M; ++j) acc = O::fma(v[j], cospi_md((2 * j + 1) * (2 * k + 1), 4 * M), acc);
                z[k] = acc;
            }
        } else {
            // u_j = (v_{2j} + i v_{M-1-2j}) exp(-i pi (4j+1) / (4M))
            V ur[M / 2], ui[M / 2];
#pragma unroll
            for (int j = 0; j < M / 2; ++j) rot(v[2 * j], v[M - 1 - 2 * j], 4 * j + 1, 4 * M, ur[j], ui[j]);
            FFT<M / 2, V>::run(ur, ui);
            // W_k = U_k exp(-i pi k / M); z_{2k} = Re W_k, z_{M-1-2k} = -Im W_k
#pragma unroll
            for (int k = 0; k < M / 2; ++k) {
                if constexpr (kPacked<V>) {
                    // -Im W_k = Im U_k (-cos(pi k / M)) + Re U_k sin(pi k / M): the
                    // negated rounding of the scalar form, with no packed negation
                    // (k = 0: -Im U_0)
                    if (k == 0) {
                        z[0] = ur[0];
                        z[M - 1] = O::neg(ui[0]);
                    } else {
                        const float c = cospi_md(k, M), s = sinpi_md(k, M);
                        z[2 * k] = O::fma(ur[k], c, O::mul(ui[k], s));
                        z[M - 1 - 2 * k] = O::fma(ui[k], -c, O::mul(ur[k], s));
                    }
                } else {
                    V wr, wi;
                    rot(ur[k], ui[k], k, M, wr, wi);
                    z[2 * k] = wr;
                    z[M - 1 - 2 * k] = -wi;
                }
            }
        }
    }
};

// Unscaled DCT-II: y_k = sum_j x_j cos(pi (2j+1) k / (2N)).
template <int N, typename V = float>
struct DCT2 {
    using O = VOps<V>;
    static __device__ __forceinline__ void run(const V (&x)[N], V (&y)[N])
    {
        V u[N / 2], v[N / 2], ye[N / 2], yo[N / 2];
#pragma unroll
        for (int j = 0; j < N / 2; ++j) {
            u[j] = O::add(x[j], x[N - 1 - j]);
            v[j] = O::sub(x[j], x[N - 1 - j]);
        }
        DCT2<N / 2, V>::run(u, ye);
        DCT4<N / 2, V>::run(v, yo);
#pragma unroll
        for (int m = 0; m < N / 2; ++m) { y[2 * m] = ye[m]; y[2 * m + 1] = yo[m]; }
    }
};
template <typename V>
struct DCT2<1, V> {
    static __device__ __forceinline__ void run(const V (&x)[1], V (&y)[1]) { y[0] = x[0]; }
};

// Unscaled DCT-III (transpose of DCT2): x_j = sum_k y_k cos(pi (2j+1) k / (2N)).
template <int N, typename V = float>
struct DCT3 {
    using O = VOps<V>;
    static __device__ __forceinline__ void run(const V (&y)[N], V (&x)[N])
    {
        V ye[N / 2], yo[N / 2], a[N / 2], b[N / 2];
#pragma unroll
        for (int m = 0; m < N / 2; ++m) { ye[m] = y[2 * m]; yo[m] = y[2 * m + 1]; }
        DCT3<N / 2, V>::run(ye, a);
        DCT4<N / 2, V>::run(yo, b);
#pragma unroll
        for (int j = 0; j < N / 2; ++j) {
            x[j] = O::add(a[j], b[j]);
            x[N - 1 - j] = O::sub(a[j], b[j]);
        }
    }
};
template <typename V>
struct DCT3<1, V> {
    static __device__ __forceinline__ void run(const V (&y)[1], V (&x)[1]) { x[0] = y[0]; }
};

template <int N, typename V = float>
__device__ __forceinline__ void scale_line(V (&x)[N], AxisScale s)
{
    using O = VOps<V>;
    x[0] = O::mul(x[0], s.s0);
#pragma unroll
    for (int k = 1; k < N; ++k) x[k] = O::mul(x[k], s.s1);
}

// Unscaled cores, used where every scale is folded into a table (the
// spectral composition of Prop. 1): CORE_FWD = G (DCT-II), CORE_INV = G^T
// (DCT-III).
constexpr int CORE_FWD = 4;
constexpr int CORE_INV = 5;

// One direction of the 2D transform along one axis of a line held in
// registers (or of two lines, V = float2); DIR may also be CORE_FWD or
// CORE_INV (no scale).
template <int N, int DIR, typename V = float>
__device__ __forceinline__ void line_op(V (&x)[N], AxisScale s)
{
    V y[N];
    if constexpr (DIR == CORE_FWD) {
        DCT2<N, V>::run(x, y);
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = y[k];
    } else if constexpr (DIR == CORE_INV) {
        DCT3<N, V>::run(x, y);
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = y[k];
    } else if constexpr (DIR == DIR_FWD) {
        DCT2<N, V>::run(x, y);
        scale_line<N, V>(y, s);
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = y[k];
    } else if constexpr (DIR == DIR_INV) {
        scale_line<N, V>(x, s);
        DCT3<N, V>::run(x, y);
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = y[k];
    } else {
        DCT2<N, V>::run(x, y);
        scale_line<N, V>(y, s);
        DCT3<N, V>::run(y, x);
    }
}

// Transform -- diagonal -- adjoint along one line (the middle factor of
// Prop. 1, Eq. 4): y = G x, y_k *= d[k], x = G^T y, unscaled cores (the
// scales of both axes are folded into d).
template <int N>
__device__ __forceinline__ void line_spectral(float (&x)[N], const float (&d)[N])
{
    float y[N];
    DCT2<N, float>::run(x, y);
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] *= d[k];
    DCT3<N, float>::run(y, x);
}

// line_spectral on two lines a and b held as plain float arrays, each with
// its own row of the diagonal: the first and last stages scalar, everything
// between packed (as line_op2).
template <int N>
__device__ __forceinline__ void line_spectral2(float (&a)[N], float (&b)[N], const float (&da)[N],
                                               const float (&db)[N])
{
    static_assert(N >= 4, "split of the first stage");
    constexpr int H = N / 2;
    float2 u[H], v[H], ye[H], yo[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        u[j] = make_float2(a[j] + a[N - 1 - j], b[j] + b[N - 1 - j]);
        v[j] = make_float2(a[j] - a[N - 1 - j], b[j] - b[N - 1 - j]);
    }
    DCT2<H, float2>::run(u, ye);
    DCT4<H, float2>::run(v, yo);
    // coefficient 2m is ye[m], 2m + 1 is yo[m]: the diagonal, then the adjoint
#pragma unroll
    for (int m = 0; m < H; ++m) {
        ye[m] = __fmul2_rn(ye[m], make_float2(da[2 * m], db[2 * m]));
        yo[m] = __fmul2_rn(yo[m], make_float2(da[2 * m + 1], db[2 * m + 1]));
    }
    float2 ea[H], ob[H];
    DCT3<H, float2>::run(ye, ea);
    DCT4<H, float2>::run(yo, ob);
#pragma unroll
    for (int j = 0; j < H; ++j) {
        a[j] = ea[j].x + ob[j].x; a[N - 1 - j] = ea[j].x - ob[j].x;
        b[j] = ea[j].y + ob[j].y; b[N - 1 - j] = ea[j].y - ob[j].y;
    }
}

// line_op on two lines a and b held as plain float arrays (for instance two
// rows loaded with 16-byte accesses): the first and the last stage run in
// scalar instructions that read or write the halves of packed pairs, so
// packing and unpacking cost no moves; everything between runs packed.
template <int N, int DIR>
__device__ __forceinline__ void line_op2(float (&a)[N], float (&b)[N], AxisScale s)
{
    static_assert(N >= 4, "split of the first stage");
    using O = VOps<float2>;
    constexpr int H = N / 2;
    float2 ye[H], yo[H];
    if constexpr (DIR == DIR_FWD || DIR == DIR_RT) {
        // even/odd split of the DCT-II: sums and differences, packed as they form
        float2 u[H], v[H];
#pragma unroll
        for (int j = 0; j < H; ++j) {
            u[j] = make_float2(a[j] + a[N - 1 - j], b[j] + b[N - 1 - j]);
            v[j] = make_float2(a[j] - a[N - 1 - j], b[j] - b[N - 1 - j]);
        }
        DCT2<H, float2>::run(u, ye);
        DCT4<H, float2>::run(v, yo);
        if constexpr (DIR == DIR_FWD) {
#pragma unroll
            for (int m = 0; m < H; ++m) {
                const float se = m == 0 ? s.s0 : s.s1;
                a[2 * m] = ye[m].x * se; b[2 * m] = ye[m].y * se;
                a[2 * m + 1] = yo[m].x * s.s1; b[2 * m + 1] = yo[m].y * s.s1;
            }
            return;
        }
        // round trip: E_n^2 between the core and its adjoint (even outputs ye,
        // odd outputs yo are exactly the DCT-III's split inputs)
        ye[0] = O::mul(ye[0], s.s0);
#pragma unroll
        for (int m = 1; m < H; ++m) ye[m] = O::mul(ye[m], s.s1);
#pragma unroll
        for (int m = 0; m < H; ++m) yo[m] = O::mul(yo[m], s.s1);
    } else {
        // scaled inputs of the DCT-III, split into even and odd, packed as they form
#pragma unroll
        for (int m = 0; m < H; ++m) {
            const float se = m == 0 ? s.s0 : s.s1;
            ye[m] = make_float2(a[2 * m] * se, b[2 * m] * se);
            yo[m] = make_float2(a[2 * m + 1] * s.s1, b[2 * m + 1] * s.s1);
        }
    }
    float2 ea[H], ob[H];
    DCT3<H, float2>::run(ye, ea);
    DCT4<H, float2>::run(yo, ob);
#pragma unroll
    for (int j = 0; j < H; ++j) {
        a[j] = ea[j].x + ob[j].x; a[N - 1 - j] = ea[j].x - ob[j].x;
        b[j] = ea[j].y + ob[j].y; b[N - 1 - j] = ea[j].y - ob[j].y;
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
