// Internal interfaces between the translation units of the bdct library.
// Host-side only declarations; no CUDA types leak into include/bdct.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#include <atomic>
#include <mutex>

#include "bdct.h"

namespace bdct {

// Per-device launch set-up of one kernel (its attributes, resident CTAs per
// SM and the SM count), computed once per device under a lock, so that host
// threads creating their first plans at the same time do not race on it;
// later launches read it without locking.
struct DeviceLaunchCache {
    std::mutex mu;
    std::atomic<bool> ready[64];
    int blocks[64];
    int sms[64];
    // init(dev, blocks, sms) runs at most once per device (again only if it
    // failed); its error is returned.
    template <class Init>
    cudaError_t get(int dev, Init &&init, int *blocks_out, int *sms_out)
    {
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!ready[dev].load(std::memory_order_acquire)) {
            std::lock_guard<std::mutex> lock(mu);
            if (!ready[dev].load(std::memory_order_relaxed)) {
                int b = 0, n = 0;
                cudaError_t e = init(dev, b, n);
                if (e != cudaSuccess) return e;
                blocks[dev] = b;
                sms[dev] = n;
                ready[dev].store(true, std::memory_order_release);
            }
        }
        *blocks_out = blocks[dev];
        *sms_out = sms[dev];
        return cudaSuccess;
    }
};

// A per-axis diagonal scale that takes one value at index 0 and another at
// every index > 0 -- every scale of Eq. 1 and of the REDFT pair has this form.
struct AxisScale {
    float s0, s1;
};

// Scales for one direction on both axes.  Forward: applied to the outputs of
// the core (Prop. 1 folds D_n into the final store).  Inverse: applied to the
// inputs of the adjoint core.  Round trip: the E_n^2 correction between the
// forward core and the adjoint core (Prop. 1 with Lambda = I).
struct DirScales {
    AxisScale h, w;
};

// Geometry of one execution call.
struct ExecGeom {
    const float *in;
    float *out;
    long long count;        // arrays (contiguous) or tiles (tiled)
    int tiled;              // 0: contiguous batch, 1: tiles of an image
    int tiles_per_row;      // tiled: img_cols / cols
    long long ld_in, ld_out;  // tiled: leading dimensions in floats
    // indexed batch (ragged classes): array a starts at in + in_off[a] and
    // out + out_off[a] (device arrays of element offsets); null = contiguous
    const long long *in_off = nullptr, *out_off = nullptr;
    // spectral direction only: the h x w diagonal (row k = frequency index
    // along h) -- folded with the scales (E Lambda E of Prop. 1) for kernels
    // that run the unscaled cores, plain Lambda for the tensor-core route
    const float *lam = nullptr;
};

// Directions of one call.  DIR_SPEC is the transform -- diagonal spectral
// operator -- inverse composition U^T Lambda U of Prop. 1 (Eq. 4).
enum Dir { DIR_FWD = 0, DIR_INV = 1, DIR_RT = 2, DIR_SPEC = 3 };

// True when the environment variable BDCT_DEBUG is set: kernel launchers then
// print their launch configuration once to stderr.
inline bool debug_enabled()
{
    static const bool on = getenv("BDCT_DEBUG") != nullptr;
    return on;
}

// ---- fp32_fused.cu
// Builds the cosine table in constant memory of the current device (FP64 on
// the GPU, rounded to FP32).  Idempotent per device.
cudaError_t fused_init_device(int device);
// True if (rows, cols) has a fused register-tile kernel.
bool fused_supported(int rows, int cols);
// `status` is the plan's device status word (bounded waits record timeouts).
cudaError_t fused_launch(int rows, int cols, Dir dir, const DirScales &sc, const ExecGeom &g,
                         unsigned int *status, cudaStream_t stream);

// ---- tma_host.cu
// A 2D tensor map (TMA) of a row-major float matrix of rows x cols with row
// stride ld floats: boxes of 32 columns x box_rows rows, 128-byte swizzle.
// CUtensorMap comes from <cuda.h>; this header only forward-declares it.
cudaError_t tma_map_2d(struct CUtensorMap_st *m, const float *base, unsigned long long rows,
                       unsigned long long cols, unsigned long long ld, int box_rows);

// ---- fp32_ring.cu
// Warp-specialized ring kernels for sides 64 and 128 (all four combinations):
// contiguous, indexed and tiled batches.
cudaError_t ring_init_table(const float *d_table);
bool ring_supported(int rows, int cols);
cudaError_t ring_launch(int rows, int cols, Dir dir, const DirScales &sc, const ExecGeom &g,
                        unsigned int *status, cudaStream_t stream);

// ---- fp32_lines.cu
// Copy the cosine table (device buffer, 4097 floats) into the line engine's
// constant memory (called by fused_init_device).
cudaError_t lines_init_table(const float *d_table);
cudaError_t lines_init_table3(const float *d_table);
// True if n has an FFT-based line engine (powers of two 64..4096, and 768).
bool lines_supported(int n);
// The line engine's twiddle tables for length n (lines_table_elems(n)
// float2 entries), generated in FP64.
size_t lines_table_elems(int n);
cudaError_t lines_gen_table(float2 *dst, int n, cudaStream_t s);
// One separable pass over `count` arrays of rows x n: every row (length n)
// gets the 1D transform of `dir` with per-index scales `sc` (forward: output
// scale, inverse: input scale, round trip: the E^2 correction), and the
// result is written transposed: dst[b][k][r] = row r's output k, arrays of
// n x rows.  Two such passes give the 2D transform in natural layout.
cudaError_t lines_pass(const float *src, float *dst, int rows, int n, long long count, Dir dir,
                       AxisScale sc, const float2 *tw, unsigned int *status, cudaStream_t stream,
                       const long long *src_off = nullptr, const long long *dst_off = nullptr,
                       bool reverse = false);

// ---- tc_split.cu
// Split-BF16 tcgen05 route for square sides 16, 32, 64.
bool tc_supported(int rows, int cols);
// BF16 elements of one operator's term table (three terms of n x n).
size_t tc_table_elems(int n);
// Split the FP64 operator matrix of (direction 1 fwd / 2 inv, norm) into three
// BF16 terms in the tensor-core B layout.
cudaError_t tc_gen_tables(__nv_bfloat16 *dst, int n, int direction, int norm, cudaStream_t s);
// `ops` holds one table (forward or inverse) or two adjacent (round trip:
// orthonormal forward, then orthonormal inverse); terms = 3, 2 or 1.
cudaError_t tc_launch(int n, Dir dir, int terms, const ExecGeom &g, const __nv_bfloat16 *ops,
                      unsigned int *status, cudaStream_t stream);

// ---- spectral.cu
// Build the plan's spectral tables from a device copy of Lambda (FP64, h x w):
// plain[k][l] = Lambda[k][l] and fold[k][l] = e_h[k] Lambda[k][l] e_w[l] with
// e_n = the squared scales of Eq. 1 (1/n at index 0, 2/n elsewhere), both
// rounded once to FP32.
cudaError_t spectral_gen_tables(const double *lam, float *plain, float *fold, int h, int w, cudaStream_t s);

// Copy `count` contiguous h x w arrays from src into the call's OUTPUT
// geometry g (contiguous or indexed through out_off).
cudaError_t copy_arrays(const float *src, const ExecGeom &g, int h, int w, cudaStream_t s);

// ---- range.cu
// Range protection: per array, the binary exponent e of its largest magnitude
// (maxbits: one word per array, cleared here), and out = in * 2^-e (the
// call's geometry, in place allowed); range_postscale multiplies the output
// by 2^e again.
cudaError_t range_prescale(const ExecGeom &g, int h, int w, unsigned int *maxbits, cudaStream_t s);
cudaError_t range_postscale(const ExecGeom &g, int h, int w, const unsigned int *maxbits, cudaStream_t s);

// ---- tc_gemm.cu
// Split-BF16 tensor-core separable passes: any side 16, 32 or a multiple of
// 64 up to 8192 per axis, and 8 x 8 arrays as one 64 x 64 Kronecker product.
bool tg_axis_ok(int n);
// BF16 elements of one blocked operator table of side n (64 for Kronecker).
size_t tg_table_elems(int n);
// Split the FP64 operator of (direction 1 fwd / 2 inv, norm) of side n (or
// the 8 x 8 Kronecker operator) into three BF16 terms, blocked for tg_pass.
cudaError_t tg_gen_table(__nv_bfloat16 *dst, int n, int direction, int norm, bool kron, cudaStream_t s);
// One pass over `count` arrays of R rows of length K: every row gets the 1D
// operator (K x K) and the result is written transposed, dst[b][n][r]
// (arrays of K x R; R = 1 writes dst[b][n]).  src_off / dst_off index the
// arrays (element offsets) or are null for contiguous arrays; lam, if not
// null, multiplies output (n, r) by lam[n * R + r].  src != dst.
// Long contractions (K a multiple of 128) first split the input into
// abuf (tg_split_elems(count * R, K) BF16 elements of plan workspace), then
// run the warp-specialized kernel; shorter ones split in the kernel (abuf
// unused, may be null).
cudaError_t tg_pass(const float *src, float *dst, const long long *src_off, const long long *dst_off, long long count,
                    int R, int K, const __nv_bfloat16 *ops, int terms, const float *lam, __nv_bfloat16 *abuf,
                    unsigned int *status, cudaStream_t stream);
size_t tg_split_elems(long long rows, int K);

// ---- dense_passes.cu
// Separable dense passes through a workspace, any shape.  `op_h`, `op_w` are
// the h x h and w x w FP32 operator matrices of one direction (scales folded
// in); the result is op_h X op_w^T for every array.
cudaError_t dense_gen_operator(float *op, int n, int direction, int norm, cudaStream_t stream);
cudaError_t dense_pass_rows(const float *in, float *out, const float *op_w, int rows_total, int w,
                            cudaStream_t stream);
cudaError_t dense_pass_cols(const float *in, float *out, const float *op_h, int h, int w,
                            long long count, cudaStream_t stream);
// Indexed variants: array b of the batch at base + off[b] (element offsets).
cudaError_t dense_pass_rows_indexed(const float *in, const long long *in_off, float *out, const float *op_w, int h,
                                    int w, long long count, cudaStream_t stream);
cudaError_t dense_pass_rows_out_indexed(const float *in, float *out, const long long *out_off, const float *op_w,
                                        int h, int w, long long count, cudaStream_t stream);
cudaError_t dense_pass_cols_indexed(const float *in, float *out, const long long *out_off, const float *op_h, int h,
                                    int w, long long count, cudaStream_t stream);

}  // namespace bdct
