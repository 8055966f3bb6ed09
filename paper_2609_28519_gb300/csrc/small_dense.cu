// On-chip dense route for small arrays of any side up to 64 that the fused
// kernels do not cover (non-power-of-two sides such as 24, 26, 40 or 48).
//
// What is computed: Eq. 2 of the BRiDCT paper as the sandwich M_h X M_w^T
// with the FP32 operator tables of the dense route (M = Q_n forward, Q_n^T
// inverse, Eq. 1; Section 7.1 makes h and w independent); the round trip is
// the forward pair then the inverse pair of the orthonormal operators
// (Prop. 1 with Lambda = I), and the spectral direction puts Lambda between
// them (Eq. 4).  A direct evaluation costs n multiply-adds per point and
// pass (Section 1.2); for n <= 64 that is arithmetic the GPU does at about
// HBM speed, so the arrays are read once and written once and every pass
// runs in shared memory -- the two-pass route through a workspace in HBM
// moves twice the bytes per pass and launches two GEMMs per chunk.
//
// Organization: persistent CTAs of 256 threads; each iteration transforms
// G arrays held in a shared buffer (rows padded to a multiple of 4 and a
// pitch of 4 mod 32 floats, padding zero), running the passes between two
// buffers and writing the last pass straight to global memory, while the
// next G arrays arrive in a third buffer by 16-byte cp.async copies.  Each thread computes
// 4 x 4 output tiles (four consecutive rows, four consecutive columns): a
// step of four contraction indices reads four float4 of the input and four
// of the operator (staged once per CTA, zero-padded; transposed for passes
// along w so that the lanes of a warp read consecutive float4) for 64
// fused multiply-adds, issued as 32 packed (two-column) instructions.  Sums of more than 16 terms are taken in blocks of
// 16 added to the running total, as in the dense route.
#include <cuda_runtime.h>

#include <cstdio>

#include "bdct_internal.h"
#include "ptx.cuh"
#include "small_dense.h"

namespace bdct {

namespace {

constexpr int kSmThreads = 256;
constexpr int kSmMaxSide = 64;
constexpr int kSmMaxPasses = 4;

struct SmallParams {
    const float *in;
    float *out;
    const long long *in_off, *out_off;  // indexed arrays (element offsets), or null
    int tpr;                            // image tiles: tiles per image row (0: arrays)
    long long ld_in, ld_out;            // image tiles: leading dimensions (floats)
    long long count;
    int h, w;
    int hp, wp;      // sides padded to a multiple of 4
    int pitch;       // buffer row pitch (floats): >= wp, 4 mod 32
    int G;           // arrays per iteration
    int npass;
    int axis[kSmMaxPasses];          // 0: along w (every row), 1: along h (every column)
    int op_at[kSmMaxPasses];         // offset (floats) of each pass's staged operator
    const float *op[kSmMaxPasses];   // n x n row-major, y = M x, scales folded in
    const float *lam;                // spectral: Lambda (h x w) after the second pass, or null
};

__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }

// Row pitch of 4 mod 32 floats (>= n): the float4 rows read by the lanes of a
// quarter-warp fall on distinct bank groups.
__host__ __device__ inline int pitch4(int n)
{
    int p = pad4(n);
    while (p % 32 != 4) p += 4;
    return p;
}

// First element and row stride of array (or image tile) a.
__device__ __forceinline__ const float *in_array(const SmallParams &p, long long a, long long &ld)
{
    if (p.tpr) {
        ld = p.ld_in;
        return p.in + (a / p.tpr) * p.h * p.ld_in + (a % p.tpr) * p.w;
    }
    ld = p.w;
    return p.in_off ? p.in + p.in_off[a] : p.in + a * (long long)p.h * p.w;
}
__device__ __forceinline__ float *out_array(const SmallParams &p, long long a, long long &ld)
{
    if (p.tpr) {
        ld = p.ld_out;
        return p.out + (a / p.tpr) * p.h * p.ld_out + (a % p.tpr) * p.w;
    }
    ld = p.w;
    return p.out_off ? p.out + p.out_off[a] : p.out + a * (long long)p.h * p.w;
}

// acc (two columns) += s * v, one packed instruction for both columns.
__device__ __forceinline__ float2 fma2s(float s, float2 v, float2 acc)
{
    return __ffma2_rn(make_float2(s, s), v, acc);
}

// One pass from buffer `src` to buffer `dst` (or, for the last pass, to the
// arrays in global memory).  Along w: dst[i][l] = sum_j src[i][j] Mt[j][l]
// (Mt = M^T staged, n = w); along h: dst[k][l] = sum_i M[k][i] src[i][l]
// (n = h).  Tiles: 4 rows x 4 columns, rt over the row tiles of all the
// iteration's arrays, lt over the column tiles; the four columns of a tile
// accumulate as two packed pairs.
template <int AXIS, bool FINAL>
__device__ __forceinline__ void small_pass(const SmallParams &p, const float *op_s, const float *src, float *dst,
                                           long long a0, int na)
{
    const int hp = p.hp, wp = p.wp, pitch = p.pitch;
    const int W4 = wp >> 2, H4 = hp >> 2;
    const int n = AXIS == 0 ? wp : hp;  // padded contraction length (a multiple of 4)
    const int tiles = na * H4 * W4;
    // stride between consecutive contraction rows of the operand read per q
    const int qstride = AXIS == 0 ? wp : pitch;
    for (int t = threadIdx.x; t < tiles; t += kSmThreads) {
        const int lt = t % W4, rt = t / W4;  // rt = a * H4 + row tile
        const int a = rt / H4, r0 = (rt - a * H4) * 4;
        const float *sa = src + (size_t)a * hp * pitch;
        // rp: the four rows read along the contraction (input rows along w,
        // operator rows along h); qp: the operand read four columns wide
        const float *rp = AXIS == 0 ? sa + r0 * pitch : op_s + r0 * hp;
        const int rstride = AXIS == 0 ? pitch : hp;
        const float *qp = AXIS == 0 ? op_s + 4 * lt : sa + 4 * lt;
        float2 acc[4][2];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r][0] = acc[r][1] = make_float2(0.0f, 0.0f);
        for (int k0 = 0; k0 < n; k0 += 16) {
            float2 part[4][2];
#pragma unroll
            for (int r = 0; r < 4; ++r) part[r][0] = part[r][1] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int s4 = 0; s4 < 16; s4 += 4) {
                const int k = k0 + s4;
                if (k < n) {
                    float4 rv[4], qv[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) rv[r] = *reinterpret_cast<const float4 *>(rp + r * rstride + k);
#pragma unroll
                    for (int q = 0; q < 4; ++q) qv[q] = *reinterpret_cast<const float4 *>(qp + (k + q) * qstride);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const float rs[4] = {rv[r].x, rv[r].y, rv[r].z, rv[r].w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            part[r][0] = fma2s(rs[q], make_float2(qv[q].x, qv[q].y), part[r][0]);
                            part[r][1] = fma2s(rs[q], make_float2(qv[q].z, qv[q].w), part[r][1]);
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                acc[r][0] = __fadd2_rn(acc[r][0], part[r][0]);
                acc[r][1] = __fadd2_rn(acc[r][1], part[r][1]);
            }
        }
        if constexpr (FINAL) {
            // rows r0.. of array a0 + a, columns 4 lt.. (w is a multiple of 4)
            long long ld;
            float *g = out_array(p, a0 + a, ld);
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r0 + r < p.h)
                    *reinterpret_cast<float4 *>(g + (long long)(r0 + r) * ld + 4 * lt) =
                        make_float4(acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y);
        } else {
            // padding rows (h not a multiple of 4) are stored as zeros, not as
            // their sums: a non-finite input would make those 0 * inf = NaN,
            // and the buffer goes on to hold the CTA's later arrays, whose
            // sums take the padding rows in with zero weights (0 * NaN)
            float *da = dst + (size_t)a * hp * pitch;
#pragma unroll
            for (int r = 0; r < 4; ++r)
                *reinterpret_cast<float4 *>(da + (r0 + r) * pitch + 4 * lt) =
                    r0 + r < p.h ? make_float4(acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y)
                                 : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
}

// Issue the 16-byte asynchronous copies of arrays a0 .. a0 + na - 1 into
// buffer `dst` (this thread's share).  Thread t copies chunk t mod q4 of the
// group's rows t / q4, t / q4 + R, ... (R = 256 / q4 rows per sweep), its
// array and row advanced incrementally rather than divided out per copy.
__device__ __forceinline__ void small_fill(const SmallParams &p, float *dst, long long a0, int na)
{
    const int q4 = p.w >> 2, R = kSmThreads / q4;
    const int c4 = threadIdx.x % q4, r_start = threadIdx.x / q4;
    if (r_start < R) {
        const int da = R / p.h, di = R - da * p.h;
        int a = r_start / p.h, i = r_start - a * p.h;
        for (int row = r_start; row < na * p.h; row += R) {
            long long ld;
            const float *g = in_array(p, a0 + a, ld);
            cp_async16(dst + ((size_t)a * p.hp + i) * p.pitch + 4 * c4, g + (long long)i * ld + 4 * c4);
            i += di;
            a += da;
            if (i >= p.h) {
                i -= p.h;
                ++a;
            }
        }
    }
    cp_async_commit();
}

template <int AXIS>
__device__ __forceinline__ void small_pass_any(const SmallParams &p, bool final_pass, const float *op_s,
                                               const float *src, float *dst, long long a0, int na)
{
    if (final_pass) small_pass<AXIS, true>(p, op_s, src, dst, a0, na);
    else small_pass<AXIS, false>(p, op_s, src, dst, a0, na);
}

__global__ void __launch_bounds__(kSmThreads) k_small_dense(const SmallParams p)
{
    extern __shared__ __align__(16) float ssm[];
    const int hp = p.hp, wp = p.wp, pitch = p.pitch;
    const size_t buf = (size_t)p.G * hp * pitch;
    // three buffers: the group being transformed alternates between two of
    // them, the next group loads into the third
    float *bufs[3] = {ssm, ssm + buf, ssm + 2 * buf};
    float *ops = ssm + 3 * buf;
    const int tid = threadIdx.x;

    pdl_launch_dependents();
    // the operators of every pass, zero-padded: along w transposed (Mt[j][l],
    // wp x wp), along h as they are (M[k][i], hp x hp).  They are plan tables
    // written before any transform, so reading them ahead of the wait on the
    // previous kernel is safe.
    for (int q = 0; q < p.npass; ++q) {
        const int n = p.axis[q] == 0 ? p.w : p.h, np = p.axis[q] == 0 ? wp : hp;
        float *o = ops + p.op_at[q];
        for (int e = tid; e < np * np; e += kSmThreads) {
            const int r = e / np, c = e % np;
            float v = 0.0f;
            if (r < n && c < n) v = p.axis[q] == 0 ? p.op[q][(size_t)c * n + r] : p.op[q][(size_t)r * n + c];
            o[e] = v;
        }
    }
    // zero the buffers once: padding rows stay zero (the copies write only
    // the arrays' own rows, the passes zeros into the padding rows; the
    // width is a multiple of 4, so there are no padding columns)
    for (size_t e = tid; e < 3 * buf; e += kSmThreads) ssm[e] = 0.0f;
    pdl_wait_prerequisites();
    __syncthreads();

    const long long step = (long long)gridDim.x * p.G;
    long long a0 = (long long)blockIdx.x * p.G;
    int cur = 0;  // buffer holding the current group
    if (a0 < p.count) small_fill(p, bufs[cur], a0, (int)((p.count - a0) < p.G ? (p.count - a0) : p.G));
    for (; a0 < p.count; a0 += step) {
        const int na = (int)((p.count - a0) < p.G ? (p.count - a0) : p.G);
        // the next group into the buffer that is neither the current one nor
        // its partner (both free: the previous iteration ended on a barrier)
        const int nxt = (cur + 2) % 3;
        const long long an = a0 + step;
        if (an < p.count) {
            small_fill(p, bufs[nxt], an, (int)((p.count - an) < p.G ? (p.count - an) : p.G));
            cp_async_wait_group<1>();  // this group's copies have landed, the next group's may not
        } else {
            cp_async_wait_group<0>();
        }
        __syncthreads();
        float *src = bufs[cur], *dst = bufs[(cur + 1) % 3];
        for (int q = 0; q < p.npass; ++q) {
            const bool fin = q + 1 == p.npass;
            if (p.axis[q] == 0) small_pass_any<0>(p, fin, ops + p.op_at[q], src, dst, a0, na);
            else small_pass_any<1>(p, fin, ops + p.op_at[q], src, dst, a0, na);
            __syncthreads();
            if (fin) break;
            if (q == 1 && p.lam) {
                // the orthonormal spectrum times Lambda (Eq. 4)
                const int hw = p.h * p.w;
                for (int e = tid; e < na * hw; e += kSmThreads) {
                    const int a = e / hw, rem = e - a * hw, k = rem / p.w, l = rem - k * p.w;
                    dst[((size_t)a * hp + k) * pitch + l] *= p.lam[rem];
                }
                __syncthreads();
            }
            float *t = src;
            src = dst;
            dst = t;
        }
        cur = nxt;
    }
}

}  // namespace

bool small_dense_supported(int h, int w)
{
    return h >= 1 && w >= 4 && h <= kSmMaxSide && w <= kSmMaxSide && w % 4 == 0;
}

cudaError_t small_dense_run(int h, int w, int npass, const int *axis, const float *const *op, const float *lam,
                            const ExecGeom &g, cudaStream_t stream)
{
    if (!small_dense_supported(h, w) || npass < 2 || npass > kSmMaxPasses) return cudaErrorInvalidValue;
    if (g.count <= 0) return cudaSuccess;
    SmallParams p{};
    p.in = g.in;
    p.out = g.out;
    p.in_off = g.in_off;
    p.out_off = g.out_off;
    p.tpr = g.tiled ? g.tiles_per_row : 0;
    p.ld_in = g.ld_in;
    p.ld_out = g.ld_out;
    p.count = g.count;
    p.h = h;
    p.w = w;
    p.hp = pad4(h);
    p.wp = pad4(w);
    p.pitch = pitch4(w);
    p.npass = npass;
    p.lam = lam;
    int at = 0;
    for (int q = 0; q < npass; ++q) {
        p.axis[q] = axis[q];
        p.op[q] = op[q];
        p.op_at[q] = at;
        at += axis[q] == 0 ? p.wp * p.wp : p.hp * p.hp;
    }
    // arrays per iteration: the three buffers within 96 KiB, and among the
    // counts that fit, the one whose output tiles fill the 256 threads best
    // (a pass takes ceil(tiles / 256) tile times), the larger on a tie
    const int tiles1 = (p.hp / 4) * (p.wp / 4);
    const size_t arr_bytes = (size_t)p.hp * p.pitch * sizeof(float);
    int gmax = (int)((96 * 1024) / (3 * arr_bytes));
    if (gmax < 1) gmax = 1;
    if (gmax > 64) gmax = 64;
    int G = 1;
    double best = 0.0;
    for (int c = 1; c <= gmax; ++c) {
        const int tiles = c * tiles1;
        const double fill = (double)tiles / (kSmThreads * ((tiles + kSmThreads - 1) / kSmThreads));
        if (fill >= best - 1e-9) {
            best = fill;
            G = c;
        }
    }
    p.G = G;
    const size_t smem = ((size_t)3 * G * p.hp * p.pitch + (size_t)at) * sizeof(float);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;

    static DeviceLaunchCache cache;
    int dev = 0, bps = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cache.get(
        dev,
        [&](int d, int &b, int &n) {
            cudaError_t r = cudaFuncSetAttribute(k_small_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 227 * 1024);
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
            b = 1;
            return r;
        },
        &bps, &sms);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_dense, kSmThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long groups = (p.count + G - 1) / G;
    long long grid = (long long)per_sm * sms;
    if (grid > groups) grid = groups;
    if (debug_enabled()) {
        // once per configuration, not per launch
        static std::mutex mu;
        static long long last = -1;
        const long long key = ((long long)h << 20) | ((long long)w << 8) | npass;
        std::lock_guard<std::mutex> lock(mu);
        if (key != last) {
            last = key;
            fprintf(stderr, "[bdct] k_small_dense %dx%d: %d passes, %d arrays per iteration, %d CTAs/SM, smem %zu B\n",
                    h, w, npass, G, per_sm, smem);
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kSmThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_small_dense, p);
}

}  // namespace bdct
