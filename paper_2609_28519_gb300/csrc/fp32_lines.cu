// FFT-based FP32 line engine: one separable pass of the 2D DCT for long
// lines (64 .. 4096 points, powers of two, and 768 = 2 * 3 * 2^7).
//
// What is computed: the 1D factor of Eq. 2 of the BRiDCT paper along every
// row of a batch of arrays -- y_k = s_k sum_j x_j cos(pi (2j+1) k / (2N))
// (forward), its adjoint x_j = sum_k s_k y_k cos(...) (inverse), or the
// forward, the E_n^2 correction and the adjoint (round trip, Prop. 1) -- with
// the result written transposed, so that two passes (rows, then the rows of
// the transposed intermediate) give the 2D transform in natural layout.
//
// The length-N DCT-II of a real line is evaluated exactly through a complex
// FFT of L = N/2 points (Makhoul's reordering):
//   v_i = x_{2i} (i < L),  v_{N-1-i} = x_{2i+1};   z_m = v_{2m} + i v_{2m+1};
//   Z = FFT_L(z) by the four-step method, L = L1 * L2: L2 FFTs of length L1
//   on stride-L2 subsequences, twiddles exp(-2 pi i m2 k1 / L), L1 FFTs of
//   length L2; then with E_k = (Z_k + conj Z_{L-k}) / 2,
//   O_k = (Z_k - conj Z_{L-k}) / (2i), V_k = E_k + exp(-2 pi i k / N) O_k:
//   y_k = Re(exp(-i pi k / (2N)) V_k), y_{N-k} = -Im(exp(-i pi k / (2N)) V_k).
// The DCT-III runs the same steps backwards (its 1/L folded into a factor 2
// on y_0).  Sub-FFTs (radix 2 and 3, up to 64 points) run in registers
// (dct_cores.cuh); a warp transforms one to four lines; the FFT stays within
// FP32 rounding of the exact sums (error grows like log N).
#include <cuda_runtime.h>

#include <cstdio>

#include "dct_cores.cuh"
#include "ptx.cuh"

namespace bdct {

cudaError_t lines_init_table(const float *d_table) { return init_cos_table(d_table); }
cudaError_t lines_init_table3(const float *d_table) { return init_cos_table3(d_table); }

bool lines_supported(int n)
{
    return n == 64 || n == 128 || n == 256 || n == 512 || n == 1024 || n == 2048 || n == 4096 || n == 768;
}

template <int N>
struct LineCfg {
    static constexpr int L = N / 2;
    // four-step split L = L1 * L2 (step A: FFTs of L1, step C: FFTs of L2)
    static constexpr int L1 = (N == 64) ? 4 : (N == 128) ? 8 : (N == 256) ? 8 : (N == 512) ? 16 : (N == 1024) ? 16
                            : (N == 768) ? 12 : 32;
    static constexpr int L2 = L / L1;
    static constexpr int TPL_RAW = L1 > L2 ? L1 : L2;
    static constexpr int TPL = TPL_RAW > 32 ? 32 : TPL_RAW;  // threads per line
    static constexpr int LPW = 32 / TPL;                     // lines per warp at once
    static constexpr int NW = N >= 4096 ? 4 : 8;             // warps per CTA
    static constexpr int THREADS = 32 * NW;
    static constexpr int PR = N <= 512 ? 32 : (N <= 1024 ? 16 : (N == 2048 ? 8 : 4));  // rows per panel
    static constexpr int PP = N + 2 * L1 + 2;                // panel row pitch (floats)
    static constexpr int A_FLOATS = 2 * L1 * (L2 + 1);       // step-A output, padded
    static constexpr int SCR = A_FLOATS > N ? A_FLOATS : N;  // per-line scratch (floats)
    static constexpr int ROUNDS = PR / (NW * LPW);
    static constexpr int DELTA = 16 / LPW;                   // row distance of a warp's lines
    static constexpr int SEG = PR < 16 ? PR : 16;            // rows per transposed-store segment
    static constexpr int PAIRS = (L / 2 + 1 + TPL - 1) / TPL;  // split tasks per lane
    static constexpr int TWN = N + 1;                        // quarter-wave twiddles
    static constexpr size_t SMEM = (size_t)PR * PP * 4 + (size_t)NW * LPW * SCR * 4 + (size_t)TWN * 8;
    static_assert(L1 * L2 == L && L1 <= 32, "split");
    static_assert(ROUNDS >= 1 && ROUNDS * NW * LPW == PR, "panel");
    static_assert(LPW == 1 || PR % 16 == 0, "line groups");
    static_assert((PP % 4) == 2, "row pitch 2 mod 4 floats");
};

// exp(-i pi r / (2N)) for any r, from the quarter table tw[0..N] (angles 0..pi/2).
template <int N>
__device__ __forceinline__ float2 twq(const float2 *tw, int r)
{
    r %= 4 * N;
    if (r < 0) r += 4 * N;
    bool conj = false;
    if (r > 2 * N) { r = 4 * N - r; conj = true; }  // exp(-i(2pi - a)) = conj(exp(-i a))
    float2 v;
    if (r <= N) v = tw[r];
    else {  // a = pi/2 + b: exp(-i a) = -i exp(-i b)
        const float2 t = tw[r - N];
        v = make_float2(t.y, -t.x);
    }
    return conj ? make_float2(v.x, -v.y) : v;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Step A of the four-step FFT: for every task m2 of this lane, the FFT of
// length L1 of src[L2*m1 + m2] (m1 < L1), times exp(-2 pi i m2 k1 / L),
// written to A[k1][m2] of dst (pitch L2 + 1).  src and dst are distinct.
template <int N>
__device__ __forceinline__ void step_a(const float2 *src, float2 *dst, const float2 *tw, int t)
{
    using C = LineCfg<N>;
#pragma unroll 1
    for (int m2 = t; m2 < C::L2; m2 += C::TPL) {
        float re[C::L1], im[C::L1];
#pragma unroll
        for (int m1 = 0; m1 < C::L1; ++m1) {
            const float2 v = src[C::L2 * m1 + m2];
            re[m1] = v.x;
            im[m1] = v.y;
        }
        FFT<C::L1>::run(re, im);
#pragma unroll
        for (int k1 = 0; k1 < C::L1; ++k1) {
            // exp(-2 pi i m2 k1 / L) = exp(-i pi (8 m2 k1) / (2N))
            const float2 t1 = k1 == 0 ? make_float2(1.f, 0.f) : twq<N>(tw, 8 * m2 * k1);
            dst[k1 * (C::L2 + 1) + m2] = cmul(make_float2(re[k1], im[k1]), t1);
        }
    }
}

// Step C for task k1: FFT of length L2 of A[k1][*]; Z_{k1 + L1 k2} in re/im.
template <int N>
__device__ __forceinline__ void step_c(const float2 *A, int k1, float (&re)[LineCfg<N>::L2], float (&im)[LineCfg<N>::L2])
{
    using C = LineCfg<N>;
#pragma unroll
    for (int m2 = 0; m2 < C::L2; ++m2) {
        const float2 v = A[k1 * (C::L2 + 1) + m2];
        re[m2] = v.x;
        im[m2] = v.y;
    }
    FFT<C::L2>::run(re, im);
}

// Forward DCT-II of one line.  On entry `line` holds z (Makhoul order, as
// float2); on exit y_k * s_k in natural order.
template <int N>
__device__ __forceinline__ void line_forward(float *line, float *scr, const float2 *tw, int t, AxisScale s)
{
    using C = LineCfg<N>;
    float2 *z = reinterpret_cast<float2 *>(line);
    float2 *A = reinterpret_cast<float2 *>(scr);
    step_a<N>(z, A, tw, t);  // line -> scratch
    __syncwarp();
    if (t < C::L1) {  // scratch -> Z (line, natural order)
        float re[C::L2], im[C::L2];
        step_c<N>(A, t, re, im);
#pragma unroll
        for (int k2 = 0; k2 < C::L2; ++k2) z[t + C::L1 * k2] = make_float2(re[k2], im[k2]);
    }
    __syncwarp();
    // split: every lane reads its pairs (Z_k, Z_{L-k}) first, then writes y over them
    float2 za[C::PAIRS], zb[C::PAIRS];
#pragma unroll
    for (int q = 0; q < C::PAIRS; ++q) {
        const int k = t + q * C::TPL;
        if (k <= C::L / 2) {
            za[q] = z[k];
            zb[q] = z[k == 0 ? 0 : C::L - k];
        }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < C::PAIRS; ++q) {
        const int k = t + q * C::TPL;
        if (k > C::L / 2) continue;
        if (k == 0) {
            const float2 z0 = za[q];
            line[0] = (z0.x + z0.y) * s.s0;
            line[C::L] = (z0.x - z0.y) * 0.70710678118654752f * s.s1;
            continue;
        }
        const float2 a = za[q], c = zb[q];
        const float2 E = make_float2(0.5f * (a.x + c.x), 0.5f * (a.y - c.y));
        const float2 O = make_float2(0.5f * (a.y + c.y), 0.5f * (c.x - a.x));
        const float2 P = cmul(twq<N>(tw, 4 * k), O);  // exp(-2 pi i k / N) O_k
        const float2 V = make_float2(E.x + P.x, E.y + P.y);
        const float2 WV = cmul(twq<N>(tw, k), V);      // exp(-i pi k / (2N)) V_k
        line[k] = WV.x * s.s1;
        line[N - k] = -WV.y * s.s1;
        if (k != C::L - k) {
            const float2 V2 = make_float2(E.x - P.x, -(E.y - P.y));  // V_{L-k} = conj(E - P)
            const float2 WV2 = cmul(twq<N>(tw, C::L - k), V2);
            line[C::L - k] = WV2.x * s.s1;
            line[C::L + k] = -WV2.y * s.s1;
        }
    }
    __syncwarp();
}

// Inverse DCT-III of one line.  On entry `line` holds y in natural order; on
// exit x (natural order).  Input scales s_k applied on entry.
template <int N>
__device__ __forceinline__ void line_inverse(float *line, float *scr, const float2 *tw, int t, AxisScale s)
{
    using C = LineCfg<N>;
    float2 *Zc = reinterpret_cast<float2 *>(scr);  // conj(Z), natural order
    // y -> conj(Z) (scratch)
    for (int k = t; k <= C::L / 2; k += C::TPL) {
        if (k == 0) {
            const float v0 = 2.0f * line[0] * s.s0;  // factor 2 carries 1/L
            const float vl = 1.41421356237309505f * line[C::L] * s.s1;
            const float E0 = 0.5f * (v0 + vl), O0 = 0.5f * (v0 - vl);
            Zc[0] = make_float2(E0, -O0);  // Z_0 = E0 + i O0
            continue;
        }
        const float yk = line[k] * s.s1, ynk = line[N - k] * s.s1;
        const float ylk = line[C::L - k] * s.s1, ylpk = line[C::L + k] * s.s1;
        // V_k = conj(W_k) (y_k - i y_{N-k}),  V_{L-k} likewise
        const float2 Vk = cmul(conjf2(twq<N>(tw, k)), make_float2(yk, -ynk));
        const float2 Vl = cmul(conjf2(twq<N>(tw, C::L - k)), make_float2(ylk, -ylpk));
        const float2 E = make_float2(0.5f * (Vk.x + Vl.x), 0.5f * (Vk.y - Vl.y));  // (V_k + conj V_{L-k}) / 2
        const float2 D = make_float2(0.5f * (Vk.x - Vl.x), 0.5f * (Vk.y + Vl.y));  // (V_k - conj V_{L-k}) / 2
        const float2 O = cmul(conjf2(twq<N>(tw, 4 * k)), D);                        // / exp(-2 pi i k / N)
        // Z_k = E + i O;  Z_{L-k} = conj(E) + i conj(O)
        const float2 Zk = make_float2(E.x - O.y, E.y + O.x);
        Zc[k] = conjf2(Zk);
        if (k != C::L - k) {
            const float2 Zl = make_float2(E.x + O.y, -E.y + O.x);
            Zc[C::L - k] = conjf2(Zl);
        }
    }
    __syncwarp();
    // forward four-step FFT of conj(Z): step A scratch -> line (padded)
    float2 *A = reinterpret_cast<float2 *>(line);
    step_a<N>(Zc, A, tw, t);
    __syncwarp();
    // step C: conj of the result is z = IFFT(Z) (unnormalized); then v from z, x from v
    float re[C::L2], im[C::L2];
    const bool act = t < C::L1;
    if (act) step_c<N>(A, t, re, im);
    __syncwarp();  // all of A read before x overwrites the line
    if (act) {
#pragma unroll
        for (int k2 = 0; k2 < C::L2; ++k2) {
            const int m = t + C::L1 * k2;
            // z_m = conj(result); v_{2m} = Re z_m, v_{2m+1} = Im z_m
            const float v_even = re[k2], v_odd = -im[k2];
            // x_{2i} = v_i (i < L), x_{2i+1} = v_{N-1-i}
            const int i0 = 2 * m, i1 = 2 * m + 1;
            if (i0 < C::L) line[2 * i0] = v_even; else line[2 * (N - 1 - i0) + 1] = v_even;
            if (i1 < C::L) line[2 * i1] = v_odd; else line[2 * (N - 1 - i1) + 1] = v_odd;
        }
    }
    __syncwarp();
}

struct LinesParams {
    const float *src;
    float *dst;
    int rows;            // rows per array (lines per array)
    long long nrows;     // total rows
    int npanels;
    AxisScale sc;        // forward: output scales; inverse: input scales; round trip: E^2
    const long long *src_off, *dst_off;  // indexed arrays (element offsets), or null
    const float2 *tw;    // exp(-i pi r / (2N)), r = 0..N, generated in FP64 at plan time
};

template <int N, int DIR>
__global__ void __launch_bounds__(LineCfg<N>::THREADS) k_lines(const LinesParams p)
{
    using C = LineCfg<N>;
    extern __shared__ __align__(16) float lsm[];
    float *panel = lsm;
    float *scr_all = panel + C::PR * C::PP;
    float2 *tw = reinterpret_cast<float2 *>(scr_all + C::NW * C::LPW * C::SCR);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane / C::TPL, t = lane % C::TPL;

    pdl_launch_dependents();
    pdl_wait_prerequisites();
    // quarter-wave twiddles exp(-i pi r / (2N)), r = 0 .. N, from the plan's table
    for (int r = tid; r < C::TWN; r += C::THREADS) tw[r] = p.tw[r];
    __syncthreads();

    for (int pn = blockIdx.x; pn < p.npanels; pn += gridDim.x) {
        const long long r0 = (long long)pn * C::PR;  // first global row of the panel
        const long long b = r0 / p.rows;             // its array (panels never straddle two)
        const int rr = (int)(r0 - b * p.rows);
        const float *srcb = p.src_off ? p.src + p.src_off[b] : p.src + b * (long long)N * p.rows;
        // ---- load the panel (rows r0 .. r0+PR-1), coalesced 16-byte reads
        constexpr int V4 = N / 4;
        for (int i = tid; i < C::PR * V4; i += C::THREADS) {
            const int l = i / V4, q = i % V4;
            const float4 v = __ldg(reinterpret_cast<const float4 *>(srcb + (long long)(rr + l) * N) + q);
            float *row = panel + l * C::PP;
            if constexpr (DIR == DIR_INV) {
                reinterpret_cast<float2 *>(row)[2 * q] = make_float2(v.x, v.y);
                reinterpret_cast<float2 *>(row)[2 * q + 1] = make_float2(v.z, v.w);
            } else {
                // Makhoul order: (v_{2q}, v_{2q+1}) = (x_{4q}, x_{4q+2}),
                // (v_{N-2-2q}, v_{N-1-2q}) = (x_{4q+3}, x_{4q+1})
                reinterpret_cast<float2 *>(row)[q] = make_float2(v.x, v.z);
                reinterpret_cast<float2 *>(row)[N / 2 - 1 - q] = make_float2(v.w, v.y);
            }
        }
        __syncthreads();
        // ---- transform every line of the panel
#pragma unroll 1
        for (int rd = 0; rd < C::ROUNDS; ++rd) {
            // The LPW lines a warp transforms together sit DELTA = 16 / LPW rows
            // apart: with a row pitch of 2 mod 4 floats their shared-memory
            // accesses then fall into disjoint banks.
            const int grp = rd * C::NW + warp;
            const int l = (C::LPW == 1) ? grp : (grp / C::DELTA) * 16 + (grp % C::DELTA) + sub * C::DELTA;
            float *line = panel + l * C::PP;
            float *scr = scr_all + (warp * C::LPW + sub) * C::SCR;
            if constexpr (DIR == DIR_FWD) {
                line_forward<N>(line, scr, tw, t, p.sc);
            } else if constexpr (DIR == DIR_INV) {
                line_inverse<N>(line, scr, tw, t, p.sc);
            } else {
                // round trip: forward core, E^2 correction, adjoint core
                const AxisScale one = {1.0f, 1.0f};
                line_forward<N>(line, scr, tw, t, p.sc);
                line_inverse<N>(line, scr, tw, t, one);
            }
        }
        __syncthreads();
        // ---- transposed store: dst[b][k][r] with rows r0.. (same array b)
        float *dstb = p.dst_off ? p.dst + p.dst_off[b] : p.dst + b * (long long)N * p.rows;
        // a warp instruction covers SEG rows x (32 / SEG) columns; with a row
        // pitch of 2 mod 4 floats, 16 rows x 2 columns touch all 32 banks
        for (int i = tid; i < C::PR * N; i += C::THREADS) {
            const int l = i % C::SEG, cj = i / C::SEG;
            const int k = cj % N, lb = (cj / N) * C::SEG;
            dstb[(long long)k * p.rows + rr + lb + l] = panel[(lb + l) * C::PP + k];
        }
        __syncthreads();
    }
}

template <int N, int DIR>
static cudaError_t lines_launch(const LinesParams &p0, cudaStream_t stream)
{
    using C = LineCfg<N>;
    auto kern = k_lines<N, DIR>;
    static int blocks_per_sm[64], num_sms[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (blocks_per_sm[dev] == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[dev], kern, C::THREADS, C::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm[dev] < 1) return cudaErrorInvalidConfiguration;
        if (debug_enabled())
            fprintf(stderr, "[bdct] k_lines<%d,%d>: %d CTAs/SM x %d threads, panel %d rows, smem %zu B\n", N, DIR,
                    blocks_per_sm[dev], C::THREADS, C::PR, C::SMEM);
    }
    LinesParams p = p0;
    if (p.rows % C::PR != 0) return cudaErrorInvalidValue;  // panels never straddle two arrays
    const long long np = p.nrows / C::PR;
    if (np <= 0) return cudaSuccess;
    if (np > 0x7ff00000LL) return cudaErrorInvalidValue;
    p.npanels = (int)np;
    long long grid = (long long)blocks_per_sm[dev] * num_sms[dev];
    if (grid > np) grid = np;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(C::THREADS);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int N>
static cudaError_t lines_dir(Dir dir, const LinesParams &p, cudaStream_t s)
{
    switch (dir) {
        case DIR_FWD: return lines_launch<N, DIR_FWD>(p, s);
        case DIR_INV: return lines_launch<N, DIR_INV>(p, s);
        default: return lines_launch<N, DIR_RT>(p, s);
    }
}

__global__ void k_gen_line_tw(float2 *t, int n)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    // angle pi r / (2n) in [0, pi/2], evaluated in FP64
    const double a = (double)r / (2.0 * (double)n);
    t[r] = make_float2((float)cospi(a), (float)(r == n ? -1.0 : -sinpi(a)));
    if (r == n) t[r].x = 0.0f;
}

cudaError_t lines_gen_table(float2 *dst, int n, cudaStream_t s)
{
    k_gen_line_tw<<<(n + 1 + 255) / 256, 256, 0, s>>>(dst, n);
    return cudaGetLastError();
}

cudaError_t lines_pass(const float *src, float *dst, int rows, int n, long long count, Dir dir, AxisScale sc,
                       const float2 *tw, unsigned int *status, cudaStream_t stream, const long long *src_off,
                       const long long *dst_off)
{
    (void)status;
    LinesParams p{};
    p.src = src;
    p.dst = dst;
    p.tw = tw;
    p.src_off = src_off;
    p.dst_off = dst_off;
    p.rows = rows;
    p.nrows = (long long)rows * count;
    p.sc = sc;
    switch (n) {
        case 64: return lines_dir<64>(dir, p, stream);
        case 128: return lines_dir<128>(dir, p, stream);
        case 256: return lines_dir<256>(dir, p, stream);
        case 512: return lines_dir<512>(dir, p, stream);
        case 1024: return lines_dir<1024>(dir, p, stream);
        case 2048: return lines_dir<2048>(dir, p, stream);
        case 4096: return lines_dir<4096>(dir, p, stream);
        case 768: return lines_dir<768>(dir, p, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bdct
