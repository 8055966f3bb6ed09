// FP32 fused 2D DCT kernels for small power-of-two sides (8, 16, 32).
//
// What is computed: Eq. 2 of the BRiDCT paper, C(X) = Q_h X Q_w^T (forward,
// DCT-II), C^{-1}(Y) = Q_h^T Y Q_w (inverse, DCT-III) and the round trip,
// with Q_n = D_n G_n as in Eq. 3: G_n is the unscaled cosine kernel
// G[k][j] = cos(pi (2j+1) k / (2n)) and D_n the diagonal of Eq. 1.  The
// diagonal scales are folded into the pass outputs (forward), the pass inputs
// (inverse) or between the core and its adjoint (round trip, Prop. 1).
//
// 1D cores (exact factorizations, no approximated coefficients):
//  * DCT-II of length N splits into a DCT-II of length N/2 on the sums
//    x_j + x_{N-1-j} (even outputs) and a DCT-IV of length N/2 on the
//    differences (odd outputs);
//  * DCT-III (the adjoint) reverses this: DCT-III of the even inputs, DCT-IV
//    of the odd inputs, then a sum/difference butterfly;
//  * DCT-IV of length M > 4 is a pre-twiddle of M/2 complex points, a
//    length-M/2 complex FFT (radix-2, decimation in time) and a post-twiddle;
//    M <= 4 is a direct matrix product.
// Every twiddle comes from one FP32 table c_cos[r] = cos(pi r / 8192) built
// on the GPU in FP64 at plan time; all indices fold to constants.
//
// On-chip organization (the GPU counterpart of the paper's Algorithm 1 and
// Section 3.2 padded stride): a CTA of 256 threads stages A = 256/max(h,w)
// arrays in shared memory with a row pitch of w+4 floats, so that a thread
// reading a column (pass 1) and a thread reading a row with 16-byte loads
// (pass 2) both hit 32 distinct banks.  Pass 1 gives one column per thread,
// pass 2 one row per thread; each line lives in registers while its 1D core
// runs.  HBM traffic is one coalesced 16-byte read and one 16-byte write of
// every element.
#include <cuda_runtime.h>

#include "bdct_internal.h"

namespace bdct {

static __constant__ float c_cos[4097];  // cos(pi r / 8192), r = 0..4096

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
template <int L>
struct FFT {
    static __device__ __forceinline__ void run(float (&re)[L], float (&im)[L])
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
            rot(orr[k], oi[k], 2 * k, L, tr, ti);  // exp(-2 pi i k / L)
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

// ------------------------------------------------------------ kernel
constexpr int kThreads = 256;

template <int H, int W>
struct SmallGeom {
    static constexpr int LMAX = H > W ? H : W;
    static constexpr int A = kThreads / LMAX;          // arrays per CTA
    static constexpr int RP = W + 4;                   // row pitch (floats)
    static constexpr int AP = H * RP + (W < 32 ? W : 0);  // array pitch (floats)
    static constexpr int SMEM_FLOATS = A * AP;
};

template <int H, int W, int DIR, bool TILED>
__global__ void __launch_bounds__(kThreads) k_fused_small(ExecGeom g, DirScales sc)
{
    using Gm = SmallGeom<H, W>;
    constexpr int A = Gm::A, RP = Gm::RP, AP = Gm::AP;
    constexpr int HW = H * W;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);

    const int tid = threadIdx.x;
    // Arrays handled by this CTA: [first, first + n)
    long long first;
    int n;
    long long brow = 0;
    int t0 = 0;
    if constexpr (!TILED) {
        first = (long long)blockIdx.x * A;
        long long rem = g.count - first;
        n = rem < A ? (int)rem : A;
    } else {
        const int cpr = (g.tiles_per_row + A - 1) / A;
        brow = blockIdx.x / cpr;
        t0 = (int)(blockIdx.x % cpr) * A;
        int rem = g.tiles_per_row - t0;
        n = rem < A ? rem : A;
        first = 0;
    }
    if (n <= 0) return;

    // ---- load: coalesced 16-byte reads into the padded tile
    if constexpr (!TILED) {
        const float4 *src = reinterpret_cast<const float4 *>(g.in + first * HW);
        const int nvec = n * HW / 4;
        for (int q = tid; q < nvec; q += kThreads) {
            const int e = q * 4;
            const int a = e / HW, o = e % HW, r = o / W, c = o % W;
            *reinterpret_cast<float4 *>(sm + a * AP + r * RP + c) = __ldg(src + q);
        }
    } else {
        // strip of H image rows by A*W columns; columns of absent tiles skipped
        constexpr int SW = A * W;
        const float *base = g.in + (brow * H) * g.ld_in + (long long)t0 * W;
        for (int q = tid; q < H * SW / 4; q += kThreads) {
            const int e = q * 4;
            const int r = e / SW, col = e % SW, a = col / W, c = col % W;
            if (a < n)
                *reinterpret_cast<float4 *>(sm + a * AP + r * RP + c) =
                    __ldg(reinterpret_cast<const float4 *>(base + r * g.ld_in + col));
        }
    }
    __syncthreads();

    // ---- pass 1: one column per thread, 1D core along h
    if (tid < A * W) {
        const int a = tid / W, c = tid % W;
        if (a < n) {
            float x[H];
            float *p = sm + a * AP + c;
#pragma unroll
            for (int i = 0; i < H; ++i) x[i] = p[i * RP];
            line_op<H, DIR>(x, sc.h);
#pragma unroll
            for (int i = 0; i < H; ++i) p[i * RP] = x[i];
        }
    }
    __syncthreads();

    // ---- pass 2: one row per thread, 1D core along w
    if (tid < A * H) {
        const int a = tid / H, r = tid % H;
        if (a < n) {
            float x[W];
            float4 *p = reinterpret_cast<float4 *>(sm + a * AP + r * RP);
#pragma unroll
            for (int q = 0; q < W / 4; ++q) {
                float4 v = p[q];
                x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
            }
            line_op<W, DIR>(x, sc.w);
#pragma unroll
            for (int q = 0; q < W / 4; ++q) p[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        }
    }
    __syncthreads();

    // ---- store: coalesced 16-byte writes
    if constexpr (!TILED) {
        float4 *dst = reinterpret_cast<float4 *>(g.out + first * HW);
        const int nvec = n * HW / 4;
        for (int q = tid; q < nvec; q += kThreads) {
            const int e = q * 4;
            const int a = e / HW, o = e % HW, r = o / W, c = o % W;
            dst[q] = *reinterpret_cast<const float4 *>(sm + a * AP + r * RP + c);
        }
    } else {
        constexpr int SW = A * W;
        float *base = g.out + (brow * H) * g.ld_out + (long long)t0 * W;
        for (int q = tid; q < H * SW / 4; q += kThreads) {
            const int e = q * 4;
            const int r = e / SW, col = e % SW, a = col / W, c = col % W;
            if (a < n)
                *reinterpret_cast<float4 *>(base + r * g.ld_out + col) =
                    *reinterpret_cast<const float4 *>(sm + a * AP + r * RP + c);
        }
    }
}

// ------------------------------------------------------------ host side
__global__ void k_gen_cos_table(float *t)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > 4096) return;
    // cos(pi r / 8192) in FP64 with an exact argument; exact 0 at r = 4096.
    t[r] = (r == 4096) ? 0.0f : (float)cospi((double)r / 8192.0);
}

static bool g_table_ready[64];

cudaError_t fused_init_device(int device)
{
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_table_ready[device]) return cudaSuccess;
    float *tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, 4097 * sizeof(float));
    if (e != cudaSuccess) return e;
    k_gen_cos_table<<<(4097 + 255) / 256, 256>>>(tmp);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_cos, tmp, 4097 * sizeof(float), 0, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(tmp);
    if (e == cudaSuccess) g_table_ready[device] = true;
    return e;
}

bool fused_supported(int rows, int cols)
{
    auto ok = [](int n) { return n == 8 || n == 16 || n == 32; };
    return ok(rows) && ok(cols);
}

template <int H, int W, int DIR, bool TILED>
static cudaError_t launch_one(const DirScales &sc, const ExecGeom &g, cudaStream_t stream)
{
    using Gm = SmallGeom<H, W>;
    const size_t smem = (size_t)Gm::SMEM_FLOATS * sizeof(float);
    auto kern = k_fused_small<H, W, DIR, TILED>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    long long blocks;
    if (!TILED) blocks = (g.count + Gm::A - 1) / Gm::A;
    else {
        long long cpr = (g.tiles_per_row + Gm::A - 1) / Gm::A;
        blocks = (g.count / g.tiles_per_row) * cpr;
    }
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, kThreads, smem, stream>>>(g, sc);
    return cudaGetLastError();
}

template <int H, int W>
static cudaError_t launch_hw(Dir dir, const DirScales &sc, const ExecGeom &g, cudaStream_t s)
{
    const bool t = g.tiled != 0;
    switch (dir) {
        case DIR_FWD: return t ? launch_one<H, W, DIR_FWD, true>(sc, g, s) : launch_one<H, W, DIR_FWD, false>(sc, g, s);
        case DIR_INV: return t ? launch_one<H, W, DIR_INV, true>(sc, g, s) : launch_one<H, W, DIR_INV, false>(sc, g, s);
        default: return t ? launch_one<H, W, DIR_RT, true>(sc, g, s) : launch_one<H, W, DIR_RT, false>(sc, g, s);
    }
}

template <int H>
static cudaError_t launch_h(int cols, Dir dir, const DirScales &sc, const ExecGeom &g, cudaStream_t s)
{
    switch (cols) {
        case 8: return launch_hw<H, 8>(dir, sc, g, s);
        case 16: return launch_hw<H, 16>(dir, sc, g, s);
        case 32: return launch_hw<H, 32>(dir, sc, g, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fused_launch(int rows, int cols, Dir dir, const DirScales &sc, const ExecGeom &g,
                         cudaStream_t stream)
{
    switch (rows) {
        case 8: return launch_h<8>(cols, dir, sc, g, stream);
        case 16: return launch_h<16>(cols, dir, sc, g, stream);
        case 32: return launch_h<32>(cols, dir, sc, g, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bdct
