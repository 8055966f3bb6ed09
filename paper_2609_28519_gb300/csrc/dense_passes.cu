// Separable dense passes: the general-shape FP32 route.
//
// Eq. 2 of the BRiDCT paper is the sandwich M_h X M_w^T, with M = Q_n for the
// forward transform (Eq. 1) and M = Q_n^T for the inverse; Section 7.1 makes
// h and w independent.  Here the two 1D operators are applied as two FP32
// matrix products: every row first (T = X M_w^T), then every column
// (Y = M_h T).  A direct length-n evaluation costs n multiply-adds per point
// (Section 1.2), so this route serves shapes without a fused fast kernel --
// non-power-of-two sides such as 768 (which Eq. 1 defines for any n) and
// large whole arrays -- through a plan-owned workspace.
//
// The operator tables are generated on the GPU in FP64 (cos with the
// argument reduced exactly in integers) and rounded once to FP32.
#include <cuda_runtime.h>

#include "bdct_internal.h"
#include "dense_passes.h"

namespace bdct {

// cos(pi m / (2n)) for integer m, reduced exactly, evaluated in FP64.
__device__ double cos_half_turns(long long m, long long n)
{
    const long long d = 2 * n;  // angle = pi m / d
    long long r = m % (2 * d);
    if (r < 0) r += 2 * d;
    if (r > d) r = 2 * d - r;  // [0, d]
    double sign = 1.0;
    if (2 * r > d) { r = d - r; sign = -1.0; }  // [0, d/2]
    if (r == 0) return sign;
    if (2 * r == d) return 0.0;
    return sign * cospi((double)r / (double)d);
}

// direction 1 = forward: op[k][j] = s_k cos(pi (2j+1) k / (2n))
// direction 2 = inverse: op[j][k] = s_k cos(pi (2j+1) k / (2n))
// norm 0 (orthonormal): s_k = alpha_k of Eq. 1
// norm 1 (REDFT pair):  forward s_k = 2, inverse s_0 = 1, s_k = 2
__global__ void k_gen_operator(float *op, int n, int direction, int norm)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int k = (int)(idx / n), j = (int)(idx % n);
    double s;
    if (norm == 0) s = (k == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
    else if (direction == 1) s = 2.0;
    else s = (k == 0) ? 1.0 : 2.0;
    const double v = s * cos_half_turns((2LL * j + 1) * k, n);
    if (direction == 1) op[(size_t)k * n + j] = (float)v;
    else op[(size_t)j * n + k] = (float)v;
}

cudaError_t dense_gen_operator(float *op, int n, int direction, int norm, cudaStream_t stream)
{
    const long long total = (long long)n * n;
    k_gen_operator<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(op, n, direction, norm);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- GEMM tile
// C[b][m][n] = sum_k A[b][m][k] B[b][k][n] with arbitrary element strides.
// 64 x 64 output tile, K step 16, 256 threads, 4 x 4 outputs per thread.
struct GemmArgs {
    const float *A; long long sAb, sAm, sAk;
    const float *B; long long sBb, sBk, sBn;
    float *C; long long sCb, sCm, sCn;
    int M, N, K;
    // indexed batch: batch element b of A / B / C starts at off[b] (element offsets)
    const long long *aoff = nullptr, *boff = nullptr, *coff = nullptr;
    long long b0 = 0;  // index of this launch's first batch element in the offset arrays
    const float *lam = nullptr;  // or null: C[b][m][n] *= lam[m * N + n] as it is stored
};

__global__ void __launch_bounds__(256) k_gemm_strided(GemmArgs g)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const float *A = g.aoff ? g.A + g.aoff[g.b0 + b] : g.A + b * g.sAb;
    const float *B = g.boff ? g.B + g.boff[g.b0 + b] : g.B + b * g.sBb;
    float *C = g.coff ? g.C + g.coff[g.b0 + b] : g.C + b * g.sCb;
    const int tid = threadIdx.x;
    const int tm = (tid / 16) * 4, tn = (tid % 16) * 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < g.K; k0 += 16) {
        for (int q = tid; q < 16 * 64; q += 256) {
            // A tile: 64 (m) x 16 (k); B tile: 16 (k) x 64 (n)
            const int am = q / 16, ak = q % 16;
            const int gm = m0 + am, gk = k0 + ak;
            As[ak][am] = (gm < g.M && gk < g.K) ? A[gm * g.sAm + gk * g.sAk] : 0.0f;
            const int bk = q / 64, bn = q % 64;
            const int gk2 = k0 + bk, gn = n0 + bn;
            Bs[bk][bn] = (gk2 < g.K && gn < g.N) ? B[gk2 * g.sBk + gn * g.sBn] : 0.0f;
        }
        __syncthreads();
        // two-level summation: each K tile of 16 products is summed on its own
        // and then added to the running total, so the rounding error grows
        // like 16 + K/16 rather than K for long dot products
        float part[4][4] = {};
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][tm + i]; bb[i] = Bs[kk][tn + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) part[i][j] = fmaf(a[i], bb[j], part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + tm + i, gn = n0 + tn + j;
            if (gm < g.M && gn < g.N) C[gm * g.sCm + gn * g.sCn] = g.lam ? acc[i][j] * g.lam[gm * g.N + gn] : acc[i][j];
        }
}

static cudaError_t gemm(const GemmArgs &g, long long batch, cudaStream_t stream)
{
    if (batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
    // grid.z is limited to 65535: split long batches
    for (long long b0 = 0; b0 < batch; b0 += 65535) {
        const long long nb = (batch - b0) < 65535 ? (batch - b0) : 65535;
        GemmArgs s = g;
        if (g.aoff || g.boff || g.coff) s.b0 = g.b0 + b0;
        if (!g.aoff) s.A += b0 * g.sAb;
        if (!g.boff) s.B += b0 * g.sBb;
        if (!g.coff) s.C += b0 * g.sCb;
        dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, (unsigned)nb);
        if (grid.y > 65535) return cudaErrorInvalidConfiguration;
        k_gemm_strided<<<grid, 256, 0, stream>>>(s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Every row of a [rows_total x w] matrix times op_w^T: out[r][l] = sum_j in[r][j] op_w[l][j].
cudaError_t dense_pass_rows(const float *in, float *out, const float *op_w, int rows_total, int w,
                            cudaStream_t stream)
{
    // split the row count so that grid.y (tiles of 64 rows) stays within limits
    const int max_rows = 65535 * 64;
    for (long long r0 = 0; r0 < rows_total; r0 += max_rows) {
        const int nr = (int)((rows_total - r0) < max_rows ? (rows_total - r0) : max_rows);
        GemmArgs g{in + r0 * w, 0, w, 1, op_w, 0, 1, w, out + r0 * w, 0, w, 1, nr, w, w};
        cudaError_t e = gemm(g, 1, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Every column of `count` h x w arrays: out[b][k][l] = sum_i op_h[k][i] in[b][i][l].
cudaError_t dense_pass_cols(const float *in, float *out, const float *op_h, int h, int w,
                            long long count, cudaStream_t stream)
{
    return dense_pass_cols_lam(in, out, op_h, h, w, count, nullptr, stream);
}

cudaError_t dense_pass_cols_lam(const float *in, float *out, const float *op_h, int h, int w, long long count,
                                const float *lam, cudaStream_t stream)
{
    const long long hw = (long long)h * w;
    GemmArgs g{op_h, 0, h, 1, in, hw, w, 1, out, hw, w, 1, h, w, h};
    g.lam = lam;
    return gemm(g, count, stream);
}

// Indexed batch: rows pass reads array b at in + in_off[b] and writes the
// workspace contiguously; the columns pass reads the workspace and writes
// array b at out + out_off[b].
cudaError_t dense_pass_rows_indexed(const float *in, const long long *in_off, float *out, const float *op_w, int h,
                                    int w, long long count, cudaStream_t stream)
{
    const long long hw = (long long)h * w;
    GemmArgs g{in, 0, w, 1, op_w, 0, 1, w, out, hw, w, 1, h, w, w};
    g.aoff = in_off;
    return gemm(g, count, stream);
}

cudaError_t dense_pass_rows_out_indexed(const float *in, float *out, const long long *out_off, const float *op_w, int h,
                                        int w, long long count, cudaStream_t stream)
{
    const long long hw = (long long)h * w;
    GemmArgs g{in, hw, w, 1, op_w, 0, 1, w, out, 0, w, 1, h, w, w};
    g.coff = out_off;
    return gemm(g, count, stream);
}

cudaError_t dense_pass_cols_indexed(const float *in, float *out, const long long *out_off, const float *op_h, int h,
                                    int w, long long count, cudaStream_t stream)
{
    const long long hw = (long long)h * w;
    GemmArgs g{op_h, 0, h, 1, in, hw, w, 1, out, 0, w, 1, h, w, h};
    g.coff = out_off;
    return gemm(g, count, stream);
}

}  // namespace bdct
