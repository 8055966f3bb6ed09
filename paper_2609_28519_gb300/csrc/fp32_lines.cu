// FFT-based FP32 line engine: one separable pass of the 2D DCT for long
// lines (64 .. 4096 points, powers of two, and 192, 384, 768, 1536 =
// 3 * 2^6 .. 3 * 2^9: the half-length FFT takes one radix-3 stage).
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
// on y_0).
//
// GPU organization: T threads share a line, T dividing L1 and L2, so that in
// both FFT steps every thread runs whole register-resident sub-FFTs (radix 2
// and 3, dct_cores.cuh); the step-C results stay in registers and the split
// partner Z_{L-k}, held by thread T - t of the same line, arrives by warp
// shuffle.  All twiddles come from per-plan tables generated in FP64 and
// staged in shared memory.  The FFT stays within FP32 rounding of the exact
// sums (error grows like log N).
#include <cuda_runtime.h>

#include <cstdio>

#include "dct_cores.cuh"
#include "ptx.cuh"
#include "fp32_lines.h"

namespace bdct {

cudaError_t lines_init_table(const float *d_table) { return init_cos_table(d_table); }
cudaError_t lines_init_table3(const float *d_table) { return init_cos_table3(d_table); }

bool lines_supported(int n)
{
    return n == 64 || n == 128 || n == 256 || n == 512 || n == 1024 || n == 2048 || n == 4096 || n == 192 ||
           n == 384 || n == 768 || n == 1536;
}

// Four-step split L = N/2 = L1 * L2 (step A: L2 FFTs of length L1, step C:
// L1 FFTs of length L2) and the threads that share one line: T divides both
// L1 and L2, so in both steps every thread has whole sub-FFTs.
template <int N>
struct LineCfg {
    static constexpr int L = N / 2;
    static constexpr int L1 = N == 64 ? 4 : N == 128 ? 8 : N == 256 ? 8 : N == 512 ? 16 : N == 1024 ? 16
                            : (N == 192 || N == 384) ? 12 : N == 768 ? 24 : N == 1536 ? 48 : 32;
    static constexpr int L2 = L / L1;
    static constexpr int T = (N == 64 || N == 192 || N == 384) ? 4 : (N == 128 || N == 256 || N == 768) ? 8
                           : (N == 512 || N == 1024 || N == 1536) ? 16 : 32;
    static constexpr int JA = L2 / T;  // step-A sub-FFTs per thread
    static constexpr int JC = L1 / T;  // step-C sub-FFTs per thread
    static constexpr int LPW = 32 / T;  // lines per warp
    static constexpr int NW = 8;  // warps per CTA
    static constexpr int THREADS = 32 * NW;
    static constexpr int LPR = NW * LPW;  // lines per round
    // Rows per panel.  For T < 16 a half-warp holds several lines; they sit T
    // rows apart (rows 32 b + w + T sub of a 32-row block, w < T), which with a
    // row pitch of 2 mod 32 floats puts them 2T banks apart.  At least 8 rows,
    // so that the transposed store writes whole 32-byte sectors (4096-point
    // lines with 4-row panels wrote half sectors: 4 x 4096^2 forward 0.135 ->
    // 0.203 of HBM with 8 rows, the same eight warps per SM).
    static constexpr int PR = T < 16 ? (T == 4 ? 64 : 32) : (N <= 1536 ? 16 : 8);
    static constexpr int ROUNDS = PR / LPR;
    // With L2 >= 16 both FFT steps run in place in the line buffer: step A's
    // results are held in registers across a warp barrier and written back
    // with a 16-periodic XOR swizzle that keeps step C conflict-free, so no
    // per-line scratch is needed.  Shorter lines use a padded scratch.
    static constexpr bool INPLACE = L2 >= 16;
    static constexpr int A_FLOATS = INPLACE ? N : 2 * L1 * (L2 + 1);  // step-A output
    static constexpr int pitch(int need, int mod)
    {
        int p = need;
        while (p % 32 != mod) ++p;
        return p;
    }
    // line pitch: room for the step-A output of the inverse; 2 mod 32 floats so
    // that the transposed store (16 rows x 2 columns per warp) is conflict-free
    static constexpr int PP = pitch(A_FLOATS > N ? A_FLOATS : N, 2);
    // per-line scratch: the lines of one warp 2T banks apart
    static constexpr int SCR = INPLACE ? 0 : pitch(A_FLOATS > N ? A_FLOATS : N, (2 * T) % 32);
    static constexpr int SEG = PR < 16 ? PR : 16;  // rows per transposed-store segment (a multiple of 4)
    static constexpr int TAB_F2 = 3 * L;           // L step-A twiddles, then L float4 split twiddles
    static constexpr size_t SMEM = (size_t)PR * PP * 4 + (size_t)LPR * SCR * 4 + (size_t)TAB_F2 * 8;
    static_assert(L1 * L2 == L && L1 % T == 0 && L2 % T == 0 && 32 % T == 0, "split");
    static_assert(ROUNDS >= 1 && ROUNDS * LPR == PR, "panel");
    static_assert(T >= 16 || PR % 32 == 0, "line spacing");
    static_assert(JC * L2 <= 64, "registers held through the split");
    static_assert(SEG % 4 == 0 && THREADS % (SEG / 4) == 0 && N % (THREADS / (SEG / 4)) == 0, "store mapping");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Panel row of line `sub` of warp-slot `slot` (slot = round * NW + warp).
template <int N>
__device__ __forceinline__ int line_row(int slot, int sub)
{
    using C = LineCfg<N>;
    if constexpr (C::T < 16) return 32 * (slot / C::T) + (slot % C::T) + C::T * sub;
    else return slot * C::LPW + sub;
}

size_t lines_table_elems(int n) { return (size_t)3 * (n / 2); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 cmulc(float2 a, float2 b)  // a * conj(b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// Step A for this thread: for m2 = t + T j, the length-L1 FFT of
// src[L2 m1 + m2] (m1 < L1) times exp(-2 pi i m2 k1 / L), to A[k1][m2].
template <int N>
__device__ __forceinline__ void four_step_a(const float2 *src, float2 *A, const float2 *ta, int t)
{
    using C = LineCfg<N>;
#pragma unroll
    for (int j = 0; j < C::JA; ++j) {
        const int m2 = t + C::T * j;
        float re[C::L1], im[C::L1];
#pragma unroll
        for (int m1 = 0; m1 < C::L1; ++m1) {
            const float2 v = src[C::L2 * m1 + m2];
            re[m1] = v.x;
            im[m1] = v.y;
        }
        FFT<C::L1>::run(re, im);
        A[m2] = make_float2(re[0], im[0]);
#pragma unroll
        for (int k1 = 1; k1 < C::L1; ++k1)
            A[k1 * (C::L2 + 1) + m2] = cmul(make_float2(re[k1], im[k1]), ta[k1 * C::L2 + m2]);
    }
}

// Step C for this thread: for k1 = t + T j, the length-L2 FFT of A[k1][*];
// Z_{k1 + L1 k2} lands in zr[j][k2], zi[j][k2].
template <int N>
__device__ __forceinline__ void four_step_c(const float2 *A, int t, float (&zr)[LineCfg<N>::JC][LineCfg<N>::L2],
                                            float (&zi)[LineCfg<N>::JC][LineCfg<N>::L2])
{
    using C = LineCfg<N>;
#pragma unroll
    for (int j = 0; j < C::JC; ++j) {
        const int k1 = t + C::T * j;
#pragma unroll
        for (int m2 = 0; m2 < C::L2; ++m2) {
            const float2 v = A[k1 * (C::L2 + 1) + m2];
            zr[j][m2] = v.x;
            zi[j][m2] = v.y;
        }
        FFT<C::L2>::run(zr[j], zi[j]);
    }
}

// In-place variants (L2 >= 16).  A[k1][m2] sits at k1 L2 + (m2 XOR (k1 mod 16)).
template <int N>
__device__ __forceinline__ void four_step_a_inplace(float2 *buf, const float2 *ta, int t)
{
    using C = LineCfg<N>;
    float hr[C::JA][C::L1], hi[C::JA][C::L1];
#pragma unroll
    for (int j = 0; j < C::JA; ++j) {
        const int m2 = t + C::T * j;
#pragma unroll
        for (int m1 = 0; m1 < C::L1; ++m1) {
            const float2 v = buf[C::L2 * m1 + m2];
            hr[j][m1] = v.x;
            hi[j][m1] = v.y;
        }
        FFT<C::L1>::run(hr[j], hi[j]);
#pragma unroll
        for (int k1 = 1; k1 < C::L1; ++k1) {
            const float2 w = cmul(make_float2(hr[j][k1], hi[j][k1]), ta[k1 * C::L2 + m2]);
            hr[j][k1] = w.x;
            hi[j][k1] = w.y;
        }
    }
    __syncwarp();  // every read of the line done before A overwrites it
#pragma unroll
    for (int j = 0; j < C::JA; ++j) {
        const int m2 = t + C::T * j;
#pragma unroll
        for (int k1 = 0; k1 < C::L1; ++k1) buf[k1 * C::L2 + (m2 ^ (k1 & 15))] = make_float2(hr[j][k1], hi[j][k1]);
    }
    __syncwarp();
}

template <int N>
__device__ __forceinline__ void four_step_c_inplace(const float2 *buf, int t,
                                                    float (&zr)[LineCfg<N>::JC][LineCfg<N>::L2],
                                                    float (&zi)[LineCfg<N>::JC][LineCfg<N>::L2])
{
    using C = LineCfg<N>;
#pragma unroll
    for (int j = 0; j < C::JC; ++j) {
        const int k1 = t + C::T * j;
        const float2 *row = buf + k1 * C::L2;
        const int x = k1 & 15;
#pragma unroll
        for (int m2 = 0; m2 < C::L2; ++m2) {
            const float2 v = row[(m2 & ~15) + ((m2 & 15) ^ x)];
            zr[j][m2] = v.x;
            zi[j][m2] = v.y;
        }
        FFT<C::L2>::run(zr[j], zi[j]);
    }
    __syncwarp();  // every read of A done before the line is overwritten
}

// Forward DCT-II of one line.  On entry `line` holds z (Makhoul order, as
// float2); on exit y_k * s_k in natural order.  Z_k and its split partner
// Z_{L-k} sit in registers of threads t and T - t of the line (the same
// warp), so the partner comes by shuffle.
// With FOLD the table's exp(-i pi k / (2N)) carries the factor s_1 / 2
// (folded in when the table is staged), saving the scalings below.
template <int N, bool FOLD = false>
__device__ __forceinline__ void line_forward(float *line, float *scr, const float2 *ta, const float4 *ts, int t,
                                             int lane, AxisScale s)
{
    using C = LineCfg<N>;
    float2 *z = reinterpret_cast<float2 *>(line);
    float zr[C::JC][C::L2], zi[C::JC][C::L2];
    if constexpr (C::INPLACE) {
        four_step_a_inplace<N>(z, ta, t);
        four_step_c_inplace<N>(z, t, zr, zi);
    } else {
        float2 *A = reinterpret_cast<float2 *>(scr);
        four_step_a<N>(z, A, ta, t);
        __syncwarp();
        four_step_c<N>(A, t, zr, zi);
    }
    // the line buffer is free (its last reader passed a warp barrier).
    // The outputs k and L-k both come from Z_k and Z_{L-k} (the latter's E and O
    // are the former's with the imaginary parts negated), so one thread takes
    // both: k runs over this thread's slots with k2 < L2/2 (k < L/2); thread 0
    // also takes k = L/2, its own mirror.
    const int src = lane - t + (C::T - t) % C::T;
    // y_k and y_{N-k} of one index from its E and O and table entry
    auto put = [&](int k, float2 E, float2 O, const float4 &w) {
        const float2 P = cmul(make_float2(w.x, w.y), O);
        const float2 WV = cmul(make_float2(w.z, w.w), make_float2(E.x + P.x, E.y + P.y));
        if constexpr (FOLD) {
            // the table's second factor carries s_1 / 2 (E and O are 2E, 2O)
            line[k] = WV.x;
            line[N - k] = -WV.y;
        } else {
            line[k] = WV.x * s.s1;
            line[N - k] = -WV.y * s.s1;
        }
    };
    // E, O of index k from Z_k = (ar, ai) and its partner Z_{L-k} = (cr, ci)
    auto eo = [&](float ar, float ai, float cr, float ci, float2 &E, float2 &O) {
        if constexpr (FOLD) {
            E = make_float2(ar + cr, ai - ci);
            O = make_float2(ai + ci, cr - ar);
        } else {
            E = make_float2(0.5f * (ar + cr), 0.5f * (ai - ci));
            O = make_float2(0.5f * (ai + ci), 0.5f * (cr - ar));
        }
    };
#pragma unroll
    for (int j = 0; j < C::JC; ++j) {
#pragma unroll
        for (int k2 = 0; k2 < C::L2 / 2; ++k2) {
            // partner Z_{L-k}: thread T - t, slot (JC - 1 - j, L2 - 1 - k2); for
            // t = 0 the partner is this thread's own (JC - j) % JC or, for j = 0,
            // slot (0, (L2 - k2) % L2)
            float cr = __shfl_sync(0xffffffffu, zr[C::JC - 1 - j][C::L2 - 1 - k2], src);
            float ci = __shfl_sync(0xffffffffu, zi[C::JC - 1 - j][C::L2 - 1 - k2], src);
            constexpr int j0 = 0;
            if (t == 0) {
                if (j == 0) {
                    cr = zr[j0][(C::L2 - k2) % C::L2];
                    ci = zi[j0][(C::L2 - k2) % C::L2];
                } else {
                    cr = zr[(C::JC - j) % C::JC][C::L2 - 1 - k2];
                    ci = zi[(C::JC - j) % C::JC][C::L2 - 1 - k2];
                }
            }
            const int k = t + C::T * j + C::L1 * k2;
            const float ar = zr[j][k2], ai = zi[j][k2];
            if (k == 0) {
                line[0] = (ar + ai) * s.s0;
                line[C::L] = (ar - ai) * 0.70710678118654752f * s.s1;
                // k = L/2: thread 0, slot (0, L2/2), partnered with itself
                const float hr = zr[j0][C::L2 / 2], hi = zi[j0][C::L2 / 2];
                float2 E, O;
                eo(hr, hi, hr, hi, E, O);
                put(C::L / 2, E, O, ts[C::L / 2]);
            } else {
                float2 E, O;
                eo(ar, ai, cr, ci, E, O);
                put(k, E, O, ts[k]);
                put(C::L - k, make_float2(E.x, -E.y), make_float2(O.x, -O.y), ts[C::L - k]);
            }
        }
    }
    __syncwarp();
}
template <int N, bool FOLD = false>
__device__ __forceinline__ void line_inverse(float *line, float *scr, const float2 *ta, const float4 *ts, int t,
                                             AxisScale s)
{
    using C = LineCfg<N>;
    // conj(Z) in natural order: a scratch buffer, or (in place) registers
    // written over the line once every y has been read
    float2 *Zc = reinterpret_cast<float2 *>(C::INPLACE ? line : scr);
    float qr[C::JC][C::L2], qi[C::JC][C::L2];
    // y -> conj(Z): Z_k needs y_k, y_{N-k}, y_{L-k}, y_{L+k} and the table
    // entries k and L-k, and Z_{L-k} needs the same, so one thread takes both:
    // k runs over this thread's slots with k2 < L2/2 (k < L/2), and the second
    // half of the slot array holds Z_{L-k} (for k = 0: Z_{L/2}, its own mirror)
    const float sy = FOLD ? 1.0f : s.s1;  // with FOLD the table carries s_1 / 2
    const float hf = FOLD ? 1.0f : 0.5f;
#pragma unroll
    for (int j = 0; j < C::JC; ++j) {
#pragma unroll
        for (int k2 = 0; k2 < C::L2 / 2; ++k2) {
            const int k = t + C::T * j + C::L1 * k2;
            float2 za, zb;  // conj Z_k and conj Z_{L-k}
            if (k == 0) {
                const float v0 = 2.0f * line[0] * s.s0;  // factor 2 carries 1/L
                const float vl = 1.41421356237309505f * line[C::L] * s.s1;
                za = make_float2(0.5f * (v0 + vl), -0.5f * (v0 - vl));
                constexpr int H = C::L / 2;
                const float yh = line[H] * sy, ynh = line[N - H] * sy;
                const float4 w = ts[H];
                const float2 V = cmulc(make_float2(yh, -ynh), make_float2(w.z, w.w));
                const float2 E = make_float2(hf * (V.x + V.x), hf * (V.y - V.y));
                const float2 D = make_float2(hf * (V.x - V.x), hf * (V.y + V.y));
                const float2 O = cmulc(D, make_float2(w.x, w.y));
                zb = make_float2(E.x - O.y, -(E.y + O.x));
            } else {
                const float yk = line[k] * sy, ynk = line[N - k] * sy;
                const float ylk = line[C::L - k] * sy, ylpk = line[C::L + k] * sy;
                const float4 w = ts[k], wl = ts[C::L - k];
                // V_k = conj(W_k) (y_k - i y_{N-k}), V_{L-k} likewise
                const float2 Vk = cmulc(make_float2(yk, -ynk), make_float2(w.z, w.w));
                const float2 Vl = cmulc(make_float2(ylk, -ylpk), make_float2(wl.z, wl.w));
                const float2 E = make_float2(hf * (Vk.x + Vl.x), hf * (Vk.y - Vl.y));
                const float2 D = make_float2(hf * (Vk.x - Vl.x), hf * (Vk.y + Vl.y));
                const float2 O = cmulc(D, make_float2(w.x, w.y));  // / exp(-2 pi i k / N)
                za = make_float2(E.x - O.y, -(E.y + O.x));         // conj(E + i O)
                // for L-k the two V swap: E -> (E.x, -E.y), D -> (-D.x, D.y)
                const float2 Ol = cmulc(make_float2(-D.x, D.y), make_float2(wl.x, wl.y));
                zb = make_float2(E.x - Ol.y, -(Ol.x - E.y));
            }
            const int km = k == 0 ? C::L / 2 : C::L - k;
            if constexpr (C::INPLACE) {
                qr[j][k2] = za.x;
                qi[j][k2] = za.y;
                qr[j][k2 + C::L2 / 2] = zb.x;
                qi[j][k2 + C::L2 / 2] = zb.y;
            } else {
                Zc[k] = za;
                Zc[km] = zb;
            }
        }
    }
    __syncwarp();  // every read of y done before the line is overwritten
    float rr[C::JC][C::L2], ri[C::JC][C::L2];
    if constexpr (C::INPLACE) {
#pragma unroll
        for (int j = 0; j < C::JC; ++j) {
#pragma unroll
            for (int k2 = 0; k2 < C::L2 / 2; ++k2) {
                const int k = t + C::T * j + C::L1 * k2;
                Zc[k] = make_float2(qr[j][k2], qi[j][k2]);
                Zc[k == 0 ? C::L / 2 : C::L - k] = make_float2(qr[j][k2 + C::L2 / 2], qi[j][k2 + C::L2 / 2]);
            }
        }
        __syncwarp();
        four_step_a_inplace<N>(Zc, ta, t);
        four_step_c_inplace<N>(Zc, t, rr, ri);
    } else {
        float2 *A = reinterpret_cast<float2 *>(line);
        four_step_a<N>(Zc, A, ta, t);
        __syncwarp();
        four_step_c<N>(A, t, rr, ri);
    }
    __syncwarp();  // all of A read before x overwrites the line
    // z_m = conj(result): v_{2m} = Re z_m, v_{2m+1} = -Im z_m, and x_{2i} = v_i
    // (i < L), x_{2i+1} = v_{N-1-i}.  For m < L/2 the four outputs x_{4m} ..
    // x_{4m+3} are v_{2m}, v_{2m'+1}, v_{2m+1}, v_{2m'} with m' = L-1-m, whose
    // z sits in thread T-1-t at slot (JC-1-j, L2-1-k2) (k2 < L2/2 exactly when
    // m < L/2): the partner's values arrive by shuffle and the four outputs
    // leave as two 8-byte stores, taken in opposite order by the two halves of
    // each 16-lane group so that one store instruction covers distinct banks.
    const int lane = (int)(threadIdx.x & 31);
    const int src = lane - t + (C::T - 1 - t);
    const int swap = (lane >> 3) & 1;
    float2 *x2 = reinterpret_cast<float2 *>(line);
#pragma unroll
    for (int j = 0; j < C::JC; ++j) {
#pragma unroll
        for (int k2 = 0; k2 < C::L2 / 2; ++k2) {
            // each lane sends its slot (JC-1-j, L2-1-k2) and receives the partner's
            const float pe = __shfl_sync(0xffffffffu, rr[C::JC - 1 - j][C::L2 - 1 - k2], src);
            const float po = __shfl_sync(0xffffffffu, ri[C::JC - 1 - j][C::L2 - 1 - k2], src);
            const int m = t + C::T * j + C::L1 * k2;
            const float2 lo = make_float2(rr[j][k2], -po);  // x_{4m}, x_{4m+1}
            const float2 hi = make_float2(-ri[j][k2], pe);  // x_{4m+2}, x_{4m+3}
            x2[2 * m + swap] = swap ? hi : lo;
            x2[2 * m + 1 - swap] = swap ? lo : hi;
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
    const float2 *tw;    // the plan's tables for N (lines_gen_table), generated in FP64
    int reverse;         // take panels last to first (the second pass reads the
                         // intermediate the first pass wrote last, still in L2, first)
    const float *lam;    // or null: every output element (k, r) of array b is
                         // multiplied by lam[k * rows + r] as it is stored
};

template <int N, int DIR>
__global__ void __launch_bounds__(LineCfg<N>::THREADS) k_lines(const LinesParams p)
{
    using C = LineCfg<N>;
    extern __shared__ __align__(16) float lsm[];
    float *panel = lsm;
    float *scr_all = panel + C::PR * C::PP;  // per-line scratch (lines without the in-place steps)
    float2 *ta = reinterpret_cast<float2 *>(scr_all + C::LPR * C::SCR);
    const float4 *ts = reinterpret_cast<const float4 *>(ta + C::L);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane / C::T, t = lane % C::T;

    pdl_launch_dependents();
    pdl_wait_prerequisites();
    // the plan's twiddle tables (FP64-generated): step A, then the split;
    // forward and inverse fold s_1 / 2 into exp(-i pi k / (2N)) here
    constexpr bool FOLD = DIR != DIR_RT;
    const float fold = 0.5f * p.sc.s1;
    for (int r = tid; r < C::TAB_F2; r += C::THREADS) {
        float2 v = p.tw[r];
        if (FOLD && r >= C::L && ((r - C::L) & 1)) v = make_float2(v.x * fold, v.y * fold);
        ta[r] = v;
    }
    __syncthreads();

    // The panel's 16-byte chunks, ITER per thread; for lines up to 2048 points
    // the next panel's chunks are loaded into registers while the current
    // panel is transformed, so the global-load latency overlaps the work.
    constexpr int V4 = N / 4;
    constexpr int ITER = C::PR * V4 / C::THREADS;
    // (lines with a radix-3 stage hold 48 complex values through the split:
    // only the 768-point forward keeps the prefetch, measured)
    constexpr bool PREFETCH = N <= 2048 && (N % 3 != 0 || (N == 768 && DIR == DIR_FWD));
    constexpr int NB = PREFETCH ? ITER : (ITER <= 8 ? ITER : (ITER % 8 == 0 ? 8 : (ITER % 6 == 0 ? 6 : 4)));
    static_assert(ITER * C::THREADS == C::PR * V4 && ITER % NB == 0, "load batches");
    auto panel_src = [&](int pn, long long &b, int &rr) -> const float4 * {
        if (p.reverse) pn = p.npanels - 1 - pn;
        const long long r0 = (long long)pn * C::PR;  // first global row of the panel
        b = r0 / p.rows;                             // its array (panels never straddle two)
        rr = (int)(r0 - b * p.rows);
        const float *srcb = p.src_off ? p.src + p.src_off[b] : p.src + b * (long long)N * p.rows;
        return reinterpret_cast<const float4 *>(srcb + (long long)rr * N);
    };
    // chunk u of this thread -> the panel row (Makhoul order for the forward)
    auto put = [&](int i, const float4 v) {
        const int l = i / V4, q = i - l * V4;
        float2 *row = reinterpret_cast<float2 *>(panel + l * C::PP);
        if constexpr (DIR == DIR_INV) {
            row[2 * q] = make_float2(v.x, v.y);
            row[2 * q + 1] = make_float2(v.z, v.w);
        } else {
            // Makhoul order: (v_{2q}, v_{2q+1}) = (x_{4q}, x_{4q+2}),
            // (v_{N-2-2q}, v_{N-1-2q}) = (x_{4q+3}, x_{4q+1})
            row[q] = make_float2(v.x, v.z);
            row[N / 2 - 1 - q] = make_float2(v.w, v.y);
        }
    };
    float4 pre[NB];
    if constexpr (PREFETCH) {
        if (blockIdx.x < (unsigned)p.npanels) {
            long long b0;
            int r00;
            const float4 *src4 = panel_src(blockIdx.x, b0, r00);
#pragma unroll
            for (int u = 0; u < NB; ++u) pre[u] = __ldg(src4 + tid + u * C::THREADS);
        }
    }

    for (int pn = blockIdx.x; pn < p.npanels; pn += gridDim.x) {
        long long b;
        int rr;
        const float4 *src4 = panel_src(pn, b, rr);
        // ---- the panel (rows of this array), coalesced 16-byte reads
        if constexpr (PREFETCH) {
#pragma unroll
            for (int u = 0; u < NB; ++u) put(tid + u * C::THREADS, pre[u]);
            __syncthreads();
            const int nx = pn + (int)gridDim.x;
            if (nx < p.npanels) {
                long long b1;
                int r1;
                const float4 *n4 = panel_src(nx, b1, r1);
#pragma unroll
                for (int u = 0; u < NB; ++u) pre[u] = __ldg(n4 + tid + u * C::THREADS);
            }
        } else {
#pragma unroll 1
            for (int i0 = 0; i0 < ITER; i0 += NB) {
#pragma unroll
                for (int u = 0; u < NB; ++u) pre[u] = __ldg(src4 + tid + (i0 + u) * C::THREADS);
#pragma unroll
                for (int u = 0; u < NB; ++u) put(tid + (i0 + u) * C::THREADS, pre[u]);
            }
            __syncthreads();
        }
        // ---- transform every line of the panel
#pragma unroll 1
        for (int rd = 0; rd < C::ROUNDS; ++rd) {
            float *line = panel + line_row<N>(rd * C::NW + warp, sub) * C::PP;
            float *scr = scr_all + (warp * C::LPW + sub) * C::SCR;
            if constexpr (DIR == DIR_FWD) {
                line_forward<N, true>(line, scr, ta, ts, t, lane, p.sc);
            } else if constexpr (DIR == DIR_INV) {
                line_inverse<N, true>(line, scr, ta, ts, t, p.sc);
            } else {
                // round trip: forward core, E^2 correction, adjoint core
                const AxisScale one = {1.0f, 1.0f};
                line_forward<N>(line, scr, ta, ts, t, lane, p.sc);
                line_inverse<N>(line, scr, ta, ts, t, one);
            }
        }
        __syncthreads();
        // ---- transposed store: dst[b][k][r] with rows r0.. (same array b).
        // A thread writes 4 consecutive rows of one column k as one 16-byte
        // store; a warp instruction covers SEG rows x (128 / SEG) columns, and
        // with a row pitch of 2 mod 32 floats its shared-memory reads touch
        // all 32 banks.
        {
            float *dstb = p.dst_off ? p.dst + p.dst_off[b] : p.dst + b * (long long)N * p.rows;
            constexpr int SQ = C::SEG / 4;          // row quads per segment
            constexpr int KPI = C::THREADS / SQ;    // columns per step
            const int qd = tid % SQ, kk = tid / SQ;
            const long long e0 = (long long)kk * p.rows + rr + 4 * qd;  // element offset in the array
            float *g = dstb + e0;
            const long long gstep = (long long)KPI * p.rows;
#pragma unroll 1
            for (int lb = 0; lb < C::PR; lb += C::SEG) {
                const float *sp = panel + (lb + 4 * qd) * C::PP + kk;
                float *gp = g + lb;
                if (p.lam) {
                    // the spectrum times the diagonal (Prop. 1), four rows of one column
                    const float *lp = p.lam + e0 + lb;
#pragma unroll 4
                    for (int k = kk; k < N; k += KPI) {
                        const float4 l = __ldg(reinterpret_cast<const float4 *>(lp));
                        *reinterpret_cast<float4 *>(gp) =
                            make_float4(sp[0] * l.x, sp[C::PP] * l.y, sp[2 * C::PP] * l.z, sp[3 * C::PP] * l.w);
                        sp += KPI;
                        gp += gstep;
                        lp += gstep;
                    }
                } else {
#pragma unroll 4
                    for (int k = kk; k < N; k += KPI) {
                        *reinterpret_cast<float4 *>(gp) = make_float4(sp[0], sp[C::PP], sp[2 * C::PP], sp[3 * C::PP]);
                        sp += KPI;
                        gp += gstep;
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <int N, int DIR>
static cudaError_t lines_launch(const LinesParams &p0, cudaStream_t stream)
{
    using C = LineCfg<N>;
    auto kern = k_lines<N, DIR>;
    static DeviceLaunchCache cache;
    int dev = 0, blocks_per_sm = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cache.get(
        dev,
        [&](int d, int &bps, int &sms) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
            if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, C::THREADS, C::SMEM);
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
            if (r == cudaSuccess && bps < 1) r = cudaErrorInvalidConfiguration;
            if (r == cudaSuccess && debug_enabled())
                fprintf(stderr, "[bdct] k_lines<%d,%d>: %d CTAs/SM x %d threads, panel %d rows, smem %zu B\n", N, DIR,
                        bps, C::THREADS, C::PR, C::SMEM);
            return r;
        },
        &blocks_per_sm, &num_sms);
    if (e != cudaSuccess) return e;
    LinesParams p = p0;
    if (p.rows % C::PR != 0) return cudaErrorInvalidValue;  // panels never straddle two arrays
    const long long np = p.nrows / C::PR;
    if (np <= 0) return cudaSuccess;
    if (np > 0x7ff00000LL) return cudaErrorInvalidValue;
    p.npanels = (int)np;
    long long grid = (long long)blocks_per_sm * num_sms;
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

// The line engine's tables for length n (L = n / 2 = L1 * L2), in FP64 with
// the angle reduced exactly in integers:
//  [0, L):   exp(-2 pi i m2 k1 / L) at index k1 * L2 + m2 (step A);
//  [L, 3L):  for k < L the float4 (exp(-2 pi i k / n), exp(-i pi k / (2n)))
//            (the split between the half-length FFT and the DCT).
__global__ void k_gen_line_tw(float2 *t, int n, int l1)
{
    const int L = n / 2, l2 = L / l1;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < L) {
        const int k1 = r / l2, m2 = r % l2;
        const long long m = ((long long)m2 * k1) % L;  // angle -2 pi m / L
        double sn, cs;
        sincospi(-2.0 * (double)m / (double)L, &sn, &cs);
        t[r] = make_float2((float)cs, (float)sn);
    } else if (r < 2 * L) {
        const int k = r - L;
        double s1, c1, s2, c2;
        sincospi(-2.0 * (double)k / (double)n, &s1, &c1);
        sincospi(-(double)k / (2.0 * (double)n), &s2, &c2);
        float4 *q = reinterpret_cast<float4 *>(t + L);
        q[k] = make_float4((float)c1, (float)s1, (float)c2, (float)s2);
    }
}

static int line_l1(int n)
{
    switch (n) {
        case 64: return LineCfg<64>::L1;
        case 128: return LineCfg<128>::L1;
        case 256: return LineCfg<256>::L1;
        case 512: return LineCfg<512>::L1;
        case 1024: return LineCfg<1024>::L1;
        case 2048: return LineCfg<2048>::L1;
        case 4096: return LineCfg<4096>::L1;
        case 192: return LineCfg<192>::L1;
        case 384: return LineCfg<384>::L1;
        case 768: return LineCfg<768>::L1;
        case 1536: return LineCfg<1536>::L1;
        default: return 0;
    }
}

cudaError_t lines_gen_table(float2 *dst, int n, cudaStream_t s)
{
    const int l1 = line_l1(n);
    if (l1 == 0) return cudaErrorInvalidValue;
    const int total = n;  // L step-A entries + L split entries (float4, two float2 each)
    k_gen_line_tw<<<(total + 255) / 256, 256, 0, s>>>(dst, n, l1);
    return cudaGetLastError();
}

cudaError_t lines_pass(const float *src, float *dst, int rows, int n, long long count, Dir dir, AxisScale sc,
                       const float2 *tw, unsigned int *status, cudaStream_t stream, const long long *src_off,
                       const long long *dst_off, bool reverse)
{
    return lines_pass_lam(src, dst, rows, n, count, dir, sc, tw, status, stream, src_off, dst_off, reverse, nullptr);
}

cudaError_t lines_pass_lam(const float *src, float *dst, int rows, int n, long long count, Dir dir, AxisScale sc,
                           const float2 *tw, unsigned int *status, cudaStream_t stream, const long long *src_off,
                           const long long *dst_off, bool reverse, const float *lam)
{
    (void)status;
    LinesParams p{};
    p.lam = lam;
    p.reverse = reverse ? 1 : 0;
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
        case 192: return lines_dir<192>(dir, p, stream);
        case 384: return lines_dir<384>(dir, p, stream);
        case 768: return lines_dir<768>(dir, p, stream);
        case 1536: return lines_dir<1536>(dir, p, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bdct
