// FP32 ring kernels for sides 64 and 128: 64x64, 64x128, 128x64, 128x128.
//
// What is computed: Eq. 2 of the BRiDCT paper, C(X) = Q_h X Q_w^T (forward,
// DCT-II), C^{-1}(Y) = Q_h^T Y Q_w (inverse, DCT-III) and the normalized
// round trip (Prop. 1: forward core, E_n^2, adjoint core per axis), one read
// and one write of every element, both passes on chip.
//
// Organization (warp-specialized, one persistent CTA per SM):
//  * one producer warp keeps a ring of S shared-memory slots full, one array
//    per slot.  Contiguous batches and image tiles move by TMA tensor copies
//    (boxes of 32 columns x all rows, 128-byte swizzle), completing on the
//    slot's mbarrier, and leave by TMA tensor stores; the producer refills a
//    slot with the array S positions ahead once its stores have read it.
//    Indexed batches (ragged classes, arrays at arbitrary offsets) move by
//    16-byte cp.async copies placed at the same swizzled positions and leave
//    by vector stores;
//  * NG consumer groups (named barriers, no CTA-wide synchronization) take
//    the slots round robin, about three slots per group (two for the round
//    trips, which run more groups), so each group's next arrays are in
//    flight while it computes; a group transforms every row of its array,
//    then every column, in place.
//
// Slot layout (the GPU counterpart of the paper's padded stride, Section
// 3.2): columns 32b .. 32b+31 of all rows form box b; row r of a box is 128
// bytes, whose 16-byte chunk k sits at chunk position k XOR (r mod 8).  Eight
// consecutive rows at one logical chunk, and 32 consecutive columns of one
// row, then fall into distinct banks, so the row pass (one row per thread,
// 16-byte accesses) and the column pass (one column per thread) are both
// free of bank conflicts.
//
// 1D lines of 64 points run whole in one thread (dct_cores.cuh).  Lines of
// 128 points are shared by two threads of different warps through the first
// even/odd split of the DCT-II: role 0 evaluates the even outputs as a
// 64-point DCT-II of the sums x_j + x_{127-j}, role 1 the odd outputs as a
// 64-point DCT-IV of the differences.  The inverse runs the split backwards:
// role 0 a 64-point DCT-III of the even inputs (a), role 1 a 64-point DCT-IV
// of the odd inputs (b), then x_j = a_j + b_j and x_{127-j} = a_j - b_j.
// After a 128-point row pass the row is left in a permuted order that the
// column pass undoes when it writes back:
//  * forward: Y_{2m} at position m, Y_{2m+1} at 64 + ((m + 16) mod 64);
//  * inverse and round trip: x_j at j, x_{127-j} at 64 + j (j < 64);
// either way the 32 columns a warp takes in the column pass occupy 32
// distinct banks of every row.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>

#include "bdct_internal.h"
#include "dct_cores.cuh"
#include "ptx.cuh"
#include "fp32_ring.h"

namespace bdct {

cudaError_t ring_init_table(const float *d_table) { return init_cos_table(d_table); }

bool ring_supported(int rows, int cols)
{
    return (rows == 64 || rows == 128) && (cols == 64 || cols == 128);
}

constexpr int kRingMaxSmem = 232448;  // 227 KiB, the opt-in limit per CTA

// The group count depends on the direction (the kernels are instantiated per
// direction); GT, the slot and box sizes do not, and the transform helpers
// that use only those take the default.
template <int H, int W, int DIR = DIR_FWD>
struct RingCfg {
    static constexpr int TR = W / 64;   // threads per row line
    static constexpr int TC = H / 64;   // threads per column line
    static constexpr int GT = H * TR;   // threads per consumer group
    static constexpr int GW = GT / 32;  // warps per consumer group
    static constexpr int SLOT_BYTES = H * W * 4;
    static constexpr int SLOT_FLOATS = H * W;
    static constexpr int BOX_BYTES = H * 128;  // 32 columns x H rows
    // spectral direction (64 x 64 only): the folded diagonal staged once per CTA
    static constexpr int LAM_BYTES = DIR == DIR_SPEC ? H * W * 4 : 0;
    static constexpr int S_MAX = (kRingMaxSmem - 2048 - LAM_BYTES) / SLOT_BYTES;
    // about three slots per group, so that a group's next arrays load while
    // it computes; the slot count is a multiple of the group count (a group
    // always reuses slots it consumed itself, which the slot barriers' parity
    // tracking relies on)
    // (round trips, twice the arithmetic per array, run more groups over two
    // slots each: 64 x 64 seven groups, 0.67 -> 0.76 of HBM, while forward
    // and inverse measured 0.90 -> 0.81 that way; the rectangles three groups,
    // 0.26 -> 0.30 / 0.33)
    // (the spectral direction, four 1D cores per line pair like the round
    // trip plus the diagonal, runs six groups over the thirteen slots left
    // beside the diagonal, two each)
    static constexpr int NG = (H == 64 && W == 64 && DIR == DIR_RT) ? 7
                              : (H == 64 && W == 64 && DIR == DIR_SPEC) ? 6
                              : (H != W && DIR == DIR_RT)             ? 3
                                                                      : (S_MAX / 3 < 1 ? 1 : S_MAX / 3);
    static constexpr int S = (S_MAX / NG) * NG;
    static constexpr int PROD_WARP = NG * GW;
    static constexpr int THREADS = (NG * GW + 1) * 32;
    // slots start 1024-byte aligned (128-byte swizzle atoms)
    static constexpr size_t SMEM = 1024 + (size_t)S * SLOT_BYTES + (size_t)2 * S * 8 + LAM_BYTES;
    static_assert(H * TR == W * TC, "both passes use the whole group");
    static_assert(GT % 32 == 0 && S >= 2 && S % NG == 0, "ring shape");
    static_assert(SMEM <= (size_t)kRingMaxSmem, "shared memory");
    static_assert(BOX_BYTES % 1024 == 0, "swizzle atoms");
    static_assert(DIR != DIR_SPEC || (H == 64 && W == 64), "the fused spectral direction is 64 x 64 only");
};

// Named barrier over the threads of one consumer group.
__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also ANDs a predicate over the group.
__device__ __forceinline__ bool group_and(int id, int nthreads, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Slot byte offset of 16-byte chunk k (k < W/4) of row r.
template <int H>
__device__ __forceinline__ uint32_t sw_chunk(int r, int k)
{
    return (uint32_t)((k >> 3) * (H * 128) + r * 128 + (((k & 7) ^ (r & 7)) << 4));
}

// Row view: chunk k of a fixed row r is at base + (k / 8) * BOX_BYTES + o[k % 8].
struct RowView {
    uint32_t o[8];
    __device__ __forceinline__ explicit RowView(int r)
    {
#pragma unroll
        for (int t = 0; t < 8; ++t) o[t] = (uint32_t)(r * 128 + ((t ^ (r & 7)) << 4));
    }
};

// Column view: the float at slot position p of row i is at base + i * 128 + o[i % 8].
template <int H>
struct ColView {
    uint32_t o[8];
    __device__ __forceinline__ explicit ColView(int p)
    {
        const int pc = p >> 2;
#pragma unroll
        for (int t = 0; t < 8; ++t) o[t] = (uint32_t)((pc >> 3) * (H * 128) + (((pc & 7) ^ t) << 4) + (p & 3) * 4);
    }
};

template <typename T>
__device__ __forceinline__ T &at(char *base, uint32_t off)
{
    return *reinterpret_cast<T *>(base + off);
}

// Slot position of logical column c after the row pass (see the header).
template <int W, int DIR>
__device__ __forceinline__ int ring_colpos(int c)
{
    if constexpr (W == 64) return c;
    else if constexpr (DIR == DIR_FWD) return (c & 1) ? 64 + (((c >> 1) + 16) & 63) : (c >> 1);
    else return c < 64 ? c : 191 - c;
}

template <int N>
__device__ __forceinline__ void scale_from(float (&x)[N], float first, float rest)
{
    x[0] *= first;
#pragma unroll
    for (int k = 1; k < N; ++k) x[k] *= rest;
}

// Role and line of a group thread when 128-point lines are shared by two
// threads: warps alternate roles, so that each SM sub-partition (warps are
// dealt to the four sub-partitions round robin) runs one role's code only,
// and the 32 lanes of a warp take 32 consecutive lines.
__device__ __forceinline__ int role_of(int gt) { return (gt >> 5) & 1; }
__device__ __forceinline__ int line_of(int gt) { return ((gt >> 6) << 5) | (gt & 31); }

// The 64-point core of one role of a 128-point line.  On entry v holds the
// role's input (forward and round trip: sums or differences; inverse: the
// even or odd coefficients, already scaled); on exit y holds the role's
// output (forward: its coefficients, scaled; inverse and round trip: a or b).
template <int DIR>
__device__ __forceinline__ void role_core(int role, const float (&v)[64], float (&y)[64], AxisScale s)
{
    if constexpr (DIR == DIR_FWD) {
        if (role == 0) DCT2<64>::run(v, y);
        else DCT4<64>::run(v, y);
        scale_from<64>(y, role ? s.s1 : s.s0, s.s1);
    } else if constexpr (DIR == DIR_INV) {
        if (role == 0) DCT3<64>::run(v, y);
        else DCT4<64>::run(v, y);
    } else {
        float t[64];
        if (role == 0) {
            DCT2<64>::run(v, t);
            scale_from<64>(t, s.s0, s.s1);
            DCT3<64>::run(t, y);
        } else {
            DCT4<64>::run(v, t);
            scale_from<64>(t, s.s1, s.s1);
            DCT4<64>::run(t, y);
        }
    }
}

// ---------------------------------------------------------------- rectangles
// 64 x 128 and 128 x 64: the 128 side's lines are shared by two threads
// (roles), the 64 side's lines take one thread each; both passes (rows, then
// columns) run in one loop body around a single call of role_core (role 0 is
// the whole 64-point transform), so the 1D cores exist once in the code.
// LAMF (forward only): the coefficients are multiplied by the diagonal lam
// (H x W, row k = frequency along h) as the column pass stores them -- the
// first half of the spectral composition of Prop. 1 for these shapes.
template <int H, int W, int DIR, bool LAMF = false>
__device__ __forceinline__ void ring_rect(char *slot, int gt, int bar, const DirScales &sc,
                                          const float *lam = nullptr)
{
    using C = RingCfg<H, W>;
    constexpr int BB = C::BOX_BYTES;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        const AxisScale s = pass ? sc.h : sc.w;
        const bool split = pass == 0 ? W == 128 : H == 128;  // this pass's lines have 128 points
        const int role = split ? role_of(gt) : 0;
        const int ln = split ? line_of(gt) : gt;  // row (pass 0) or logical column (pass 1)
        float v[64];
        if (pass == 0) {
            const RowView rv(ln);
            if (!split) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float4 t = at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]);
                    v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
                }
            } else if (DIR == DIR_INV) {
                // role 0: even coefficients, role 1: odd coefficients
                if (role == 0) {
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const float4 t = at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]);
                        v[2 * k] = t.x; v[2 * k + 1] = t.z;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const float4 t = at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]);
                        v[2 * k] = t.y; v[2 * k + 1] = t.w;
                    }
                }
            } else {
                // sums (role 0) or differences (role 1) of x_j and x_{127-j}
                const float sg = role ? -1.0f : 1.0f;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float4 a = at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]);
                    const float4 b = at<float4>(slot, ((31 - k) >> 3) * BB + rv.o[(31 - k) & 7]);
                    v[4 * k] = fmaf(sg, b.w, a.x);
                    v[4 * k + 1] = fmaf(sg, b.z, a.y);
                    v[4 * k + 2] = fmaf(sg, b.y, a.z);
                    v[4 * k + 3] = fmaf(sg, b.x, a.w);
                }
            }
        } else {
            const ColView<H> src(ring_colpos<W, DIR>(ln));
            if (!split) {
#pragma unroll
                for (int i = 0; i < 64; ++i) v[i] = at<float>(slot, i * 128 + src.o[i & 7]);
            } else if (DIR == DIR_INV) {
                // even rows (role 0) or odd rows (role 1)
                if (role == 0) {
#pragma unroll
                    for (int m = 0; m < 64; ++m) v[m] = at<float>(slot, 2 * m * 128 + src.o[(2 * m) & 7]);
                } else {
#pragma unroll
                    for (int m = 0; m < 64; ++m) v[m] = at<float>(slot, (2 * m + 1) * 128 + src.o[(2 * m + 1) & 7]);
                }
            } else {
                const float sg = role ? -1.0f : 1.0f;
#pragma unroll
                for (int i = 0; i < 64; ++i)
                    v[i] = fmaf(sg, at<float>(slot, (127 - i) * 128 + src.o[(127 - i) & 7]),
                                at<float>(slot, i * 128 + src.o[i & 7]));
            }
        }
        if constexpr (DIR == DIR_INV) scale_from<64>(v, role ? s.s1 : s.s0, s.s1);
        // every read of the pass done before anything is overwritten (the split
        // lines' two threads share positions; the column pass of a 128-wide
        // array writes natural positions over permuted ones)
        if (split || (pass == 1 && W == 128)) group_sync(bar, C::GT);
        float y[64];
        role_core<DIR>(role, v, y, s);
        if (pass == 0) {
            const RowView rv(ln);
            if (!split || role == 0) {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]) = make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    // forward: Y_{2m+1} at 64 + ((m + 16) mod 64); inverse / round trip: b_j at 64 + j
                    const int kk = 16 + (DIR == DIR_FWD ? ((k + 4) & 15) : k);
                    at<float4>(slot, (kk >> 3) * BB + rv.o[kk & 7]) = make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]);
                }
            }
            if (DIR != DIR_FWD && split) {
                // x_j = a_j + b_j (position j), x_{127-j} = a_j - b_j (position 64 + j)
                group_sync(bar, C::GT);
                constexpr int TASKS = H * 16;  // (row, 4 consecutive j)
#pragma unroll
                for (int t = gt; t < TASKS; t += C::GT) {
                    const int rr = t >> 4, k = t & 15;
                    const uint32_t oa = sw_chunk<H>(rr, k), ob = sw_chunk<H>(rr, 16 + k);
                    const float4 a = at<float4>(slot, oa), b = at<float4>(slot, ob);
                    at<float4>(slot, oa) = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
                    at<float4>(slot, ob) = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
                }
            }
        } else {
            const ColView<H> dst(ln);
            if constexpr (LAMF) {
                // coefficient row (2m + role for split lines, m otherwise) of column ln
#pragma unroll
                for (int m = 0; m < 64; ++m) y[m] *= __ldg(lam + (split ? 2 * m + role : m) * W + ln);
            }
            if (!split) {
#pragma unroll
                for (int i = 0; i < 64; ++i) at<float>(slot, i * 128 + dst.o[i & 7]) = y[i];
            } else if (DIR == DIR_FWD) {
                // rows 2m (role 0) or 2m + 1 (role 1)
                if (role == 0) {
#pragma unroll
                    for (int m = 0; m < 64; ++m) at<float>(slot, 2 * m * 128 + dst.o[(2 * m) & 7]) = y[m];
                } else {
#pragma unroll
                    for (int m = 0; m < 64; ++m) at<float>(slot, (2 * m + 1) * 128 + dst.o[(2 * m + 1) & 7]) = y[m];
                }
            } else {
                if (role == 0) {
#pragma unroll
                    for (int j = 0; j < 64; ++j) at<float>(slot, j * 128 + dst.o[j & 7]) = y[j];  // a_j at row j
                } else {
#pragma unroll
                    for (int j = 0; j < 64; ++j)
                        at<float>(slot, (127 - j) * 128 + dst.o[(127 - j) & 7]) = y[j];  // b_j at row 127 - j
                }
                group_sync(bar, C::GT);
                // x_j = a_j + b_j, x_{127-j} = a_j - b_j; two threads per column, 32 pairs each
                auto comb = [&](int j) {
                    const uint32_t oa = j * 128 + dst.o[j & 7], ob = (127 - j) * 128 + dst.o[(127 - j) & 7];
                    const float a = at<float>(slot, oa), b = at<float>(slot, ob);
                    at<float>(slot, oa) = a + b;
                    at<float>(slot, ob) = a - b;
                };
                if (role == 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) comb(j);
                } else {
#pragma unroll
                    for (int j = 32; j < 64; ++j) comb(j);
                }
            }
        }
        group_sync(bar, C::GT);
    }
}

// ---------------------------------------------------------------- square arrays
// For h = w the two passes run in one loop, so that the 1D cores (the largest
// part of the code) exist once: pass 0 takes rows, pass 1 columns.  Same
// arithmetic, layouts and barriers as ring_rows / ring_cols.
//
// The spectral direction (64 x 64, Prop. 1 / Eq. 4 with a general diagonal)
// takes three passes with the unscaled cores: rows forward; columns forward,
// times the column's entries of the folded diagonal lam_s (E_h Lambda E_w
// with every scale of both axes in it), adjoint; rows adjoint.
template <int N, int DIR, bool LAMF = false>
__device__ __forceinline__ void ring_square(char *slot, int gt, int bar, const DirScales &sc,
                                            const float *lam_s = nullptr, const float *lam = nullptr)
{
    using C = RingCfg<N, N>;
    constexpr int BB = C::BOX_BYTES;
    constexpr int NPASS = DIR == DIR_SPEC ? 3 : 2;
#pragma unroll 1
    for (int pass = 0; pass < NPASS; ++pass) {
        const AxisScale s = (pass & 1) ? sc.h : sc.w;
        if constexpr (N == 64) {
            // one thread per line; row r (passes 0 and 2) or column c (pass 1), in place
            float x[64];
            if ((pass & 1) == 0) {
                const RowView rv(gt);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float4 t = at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]);
                    x[4 * k] = t.x; x[4 * k + 1] = t.y; x[4 * k + 2] = t.z; x[4 * k + 3] = t.w;
                }
            } else {
                const ColView<N> cv(gt);
#pragma unroll
                for (int i = 0; i < 64; ++i) x[i] = at<float>(slot, i * 128 + cv.o[i & 7]);
            }
            if constexpr (DIR == DIR_SPEC) {
                if (pass == 1) {
                    line_op<64, CORE_FWD>(x, s);
#pragma unroll
                    for (int k = 0; k < 64; ++k) x[k] *= lam_s[k * 64 + gt];
                    line_op<64, CORE_INV>(x, s);
                } else if (pass == 0) {
                    line_op<64, CORE_FWD>(x, s);
                } else {
                    line_op<64, CORE_INV>(x, s);
                }
            } else {
                line_op<64, DIR>(x, s);
            }
            if ((pass & 1) == 0) {
                const RowView rv(gt);
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]) =
                        make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
            } else {
                const ColView<N> cv(gt);
#pragma unroll
                for (int i = 0; i < 64; ++i) at<float>(slot, i * 128 + cv.o[i & 7]) = x[i];
            }
        } else {
            // two threads (roles) per 128-point line
            const int role = role_of(gt);
            const int r = line_of(gt);  // row (pass 0) or logical column (pass 1)
            float v[64];
            if (pass == 0) {
                const RowView rv(r);
                if constexpr (DIR == DIR_INV) {
                    if (role == 0) {
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            const float4 t = at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]);
                            v[2 * k] = t.x; v[2 * k + 1] = t.z;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            const float4 t = at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]);
                            v[2 * k] = t.y; v[2 * k + 1] = t.w;
                        }
                    }
                } else {
                    const float sg = role ? -1.0f : 1.0f;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float4 a = at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]);
                        const float4 b = at<float4>(slot, ((31 - k) >> 3) * BB + rv.o[(31 - k) & 7]);
                        v[4 * k] = fmaf(sg, b.w, a.x);
                        v[4 * k + 1] = fmaf(sg, b.z, a.y);
                        v[4 * k + 2] = fmaf(sg, b.y, a.z);
                        v[4 * k + 3] = fmaf(sg, b.x, a.w);
                    }
                }
            } else {
                const ColView<N> src(ring_colpos<N, DIR>(r));
                if constexpr (DIR == DIR_INV) {
                    if (role == 0) {
#pragma unroll
                        for (int m = 0; m < 64; ++m) v[m] = at<float>(slot, 2 * m * 128 + src.o[(2 * m) & 7]);
                    } else {
#pragma unroll
                        for (int m = 0; m < 64; ++m)
                            v[m] = at<float>(slot, (2 * m + 1) * 128 + src.o[(2 * m + 1) & 7]);
                    }
                } else {
                    const float sg = role ? -1.0f : 1.0f;
#pragma unroll
                    for (int i = 0; i < 64; ++i)
                        v[i] = fmaf(sg, at<float>(slot, (127 - i) * 128 + src.o[(127 - i) & 7]),
                                    at<float>(slot, i * 128 + src.o[i & 7]));
                }
            }
            if constexpr (DIR == DIR_INV) scale_from<64>(v, role ? s.s1 : s.s0, s.s1);
            group_sync(bar, C::GT);  // every read of the pass done before anything is overwritten
            float y[64];
            role_core<DIR>(role, v, y, s);
            if (pass == 0) {
                const RowView rv(r);
                if (role == 0) {
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        at<float4>(slot, (k >> 3) * BB + rv.o[k & 7]) =
                            make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int kk = 16 + (DIR == DIR_FWD ? ((k + 4) & 15) : k);
                        at<float4>(slot, (kk >> 3) * BB + rv.o[kk & 7]) =
                            make_float4(y[4 * k], y[4 * k + 1], y[4 * k + 2], y[4 * k + 3]);
                    }
                }
                if constexpr (DIR != DIR_FWD) {
                    group_sync(bar, C::GT);
                    constexpr int TASKS = N * 16;
#pragma unroll
                    for (int t = gt; t < TASKS; t += C::GT) {
                        const int rr = t >> 4, k = t & 15;
                        const uint32_t oa = sw_chunk<N>(rr, k), ob = sw_chunk<N>(rr, 16 + k);
                        const float4 a = at<float4>(slot, oa), b = at<float4>(slot, ob);
                        at<float4>(slot, oa) = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
                        at<float4>(slot, ob) = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
                    }
                }
            } else {
                const ColView<N> dst(r);
                if constexpr (LAMF) {
                    // coefficient rows 2m + role of column r, times the diagonal
#pragma unroll
                    for (int m = 0; m < 64; ++m) y[m] *= __ldg(lam + (2 * m + role) * N + r);
                }
                if constexpr (DIR == DIR_FWD) {
                    if (role == 0) {
#pragma unroll
                        for (int m = 0; m < 64; ++m) at<float>(slot, 2 * m * 128 + dst.o[(2 * m) & 7]) = y[m];
                    } else {
#pragma unroll
                        for (int m = 0; m < 64; ++m)
                            at<float>(slot, (2 * m + 1) * 128 + dst.o[(2 * m + 1) & 7]) = y[m];
                    }
                } else {
                    if (role == 0) {
#pragma unroll
                        for (int j = 0; j < 64; ++j) at<float>(slot, j * 128 + dst.o[j & 7]) = y[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < 64; ++j) at<float>(slot, (127 - j) * 128 + dst.o[(127 - j) & 7]) = y[j];
                    }
                    group_sync(bar, C::GT);
                    auto comb = [&](int j) {
                        const uint32_t oa = j * 128 + dst.o[j & 7], ob = (127 - j) * 128 + dst.o[(127 - j) & 7];
                        const float a = at<float>(slot, oa), b = at<float>(slot, ob);
                        at<float>(slot, oa) = a + b;
                        at<float>(slot, ob) = a - b;
                    };
                    if (role == 0) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) comb(j);
                    } else {
#pragma unroll
                        for (int j = 32; j < 64; ++j) comb(j);
                    }
                }
            }
        }
        group_sync(bar, C::GT);
    }
}

// ---------------------------------------------------------------- kernel
struct RingParams {
    CUtensorMap map_in, map_out;  // contiguous and tiled batches (TMA)
    const float *in;
    float *out;
    long long count;          // arrays or tiles
    int tiles_per_row;        // tiled only
    int tiled;
    int indexed;              // arrays at in + in_off[a], out + out_off[a] (cp.async path)
    long long ld_in, ld_out;  // tiled only (floats)
    DirScales sc;
    unsigned int *status;
    const long long *in_off, *out_off;
    const float *lam;         // spectral direction: the folded diagonal (H x W), else null
};

// TMA coordinates (x: column, y: row) of the first element of array or tile a.
template <int H, int W>
__device__ __forceinline__ void ring_coords(const RingParams &p, long long a, int &x, int &y)
{
    if (p.tiled) {
        const long long br = a / p.tiles_per_row, bc = a - br * p.tiles_per_row;
        x = (int)(bc * W);
        y = (int)(br * H);
    } else {
        x = 0;
        y = (int)(a * H);
    }
}

template <int H, int W, int DIR, bool LAMF = false>
__global__ void __launch_bounds__(RingCfg<H, W, DIR>::THREADS, 1) k_ring(const __grid_constant__ RingParams p)
{
    using C = RingCfg<H, W, DIR>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned slots
    const uint32_t raw = smem_u32(smem_raw);
    char *smem = reinterpret_cast<char *>(smem_raw) + (((raw + 1023u) & ~1023u) - raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::S * C::SLOT_BYTES);
    uint64_t *done = full + C::S;
    float *lam_s = reinterpret_cast<float *>(done + C::S);  // spectral only (16-byte aligned)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long grid = gridDim.x;
    const long long first = blockIdx.x;
    const int n = first < p.count ? (int)((p.count - first + grid - 1) / grid) : 0;

    if (tid == 0) {
        for (int s = 0; s < C::S; ++s) {
            mbar_init(&full[s], p.indexed ? 32 : 1);  // 32 lane arrivals (cp.async) or one expect_tx
            mbar_init(&done[s], 1);
        }
        fence_mbar_init();
    }
    pdl_launch_dependents();
    pdl_wait_prerequisites();
    if constexpr (DIR == DIR_SPEC) {
        for (int e = tid; e < H * W; e += C::THREADS) lam_s[e] = __ldg(p.lam + e);
    }
    __syncthreads();

    if (warp == C::PROD_WARP) {
        // ---------------- producer
        bool ok = true;
        int filled = 0, consumed = 0;
        if (!p.indexed) {
            // TMA tensor copies issued by lane 0
            auto fill = [&](int j) {
                const int s = j % C::S;
                char *slot = smem + s * C::SLOT_BYTES;
                int x, y;
                ring_coords<H, W>(p, first + (long long)j * grid, x, y);
                mbar_arrive_expect_tx(&full[s], (uint32_t)C::SLOT_BYTES);
#pragma unroll
                for (int b = 0; b < W / 32; ++b) tensor_load_2d(slot + b * C::BOX_BYTES, &p.map_in, x + 32 * b, y, &full[s]);
            };
            if (lane == 0) {
                const int pro = n < C::S ? n : C::S;
                for (int j = 0; j < pro; ++j) fill(j);
                filled = pro;
                for (int j = 0; j < n; ++j) {
                    const int s = j % C::S;
                    if (!mbar_wait_bounded(&done[s], (uint32_t)((j / C::S) & 1))) {
                        record_timeout(p.status);
                        ok = false;
                        break;
                    }
                    consumed = j + 1;
                    const char *slot = smem + s * C::SLOT_BYTES;
                    int x, y;
                    ring_coords<H, W>(p, first + (long long)j * grid, x, y);
#pragma unroll
                    for (int b = 0; b < W / 32; ++b) tensor_store_2d(&p.map_out, x + 32 * b, y, slot + b * C::BOX_BYTES);
                    bulk_commit();
                    // refill the slot stored one step earlier once its stores have read it
                    if (j >= 1 && j - 1 + C::S < n) {
                        bulk_wait_read<1>();
                        fill(j - 1 + C::S);
                        filled = j + C::S;
                    }
                }
                bulk_wait<0>();
            }
        } else {
            // 16-byte cp.async copies by all lanes, at the swizzled positions
            constexpr int Q = W / 4;  // chunks per row
            auto fill = [&](int j) {
                const long long a = first + (long long)j * grid;
                const int s = j % C::S;
                char *slot = smem + s * C::SLOT_BYTES;
                const float *src = p.in + p.in_off[a];
#pragma unroll 8
                for (int t = lane; t < H * Q; t += 32) {
                    const int r = t / Q, k = t - r * Q;
                    cp_async16(slot + sw_chunk<H>(r, k), src + r * W + 4 * k);
                }
                cp_async_mbar_arrive(&full[s]);
            };
            const int pro = n < C::S ? n : C::S;
            for (int j = 0; j < pro; ++j) fill(j);
            filled = pro;
            for (int j = 0; j < n; ++j) {
                const int s = j % C::S;
                ok = __all_sync(0xffffffffu, mbar_wait_bounded(&done[s], (uint32_t)((j / C::S) & 1)));
                if (!ok) {
                    if (lane == 0) record_timeout(p.status);
                    break;
                }
                consumed = j + 1;
                const long long a = first + (long long)j * grid;
                float *dst = p.out + p.out_off[a];
                const char *slot = smem + s * C::SLOT_BYTES;
#pragma unroll 8
                for (int t = lane; t < H * Q; t += 32) {
                    const int r = t / Q, k = t - r * Q;
                    *reinterpret_cast<float4 *>(dst + r * W + 4 * k) =
                        *reinterpret_cast<const float4 *>(slot + sw_chunk<H>(r, k));
                }
                __syncwarp();  // every lane's reads of the slot done before any lane refills it
                if (j + C::S < n) {
                    fill(j + C::S);
                    filled = j + C::S + 1;
                }
            }
            cp_async_wait_all();
        }
        if (!__all_sync(0xffffffffu, ok)) {
            // loads issued for arrays never consumed land (bounded) before the CTA exits
            if (lane == 0)
                for (int j = consumed; j < filled; ++j)
                    if (!mbar_wait_bounded(&full[j % C::S], (uint32_t)((j / C::S) & 1))) break;
        }
        return;
    }

    // ---------------- consumers
    const int g = warp / C::GW;
    const int gt = tid - g * C::GT;
    const int bar = 1 + g;
    for (int j = g; j < n; j += C::NG) {
        const int s = j % C::S;
        bool ok = mbar_wait_bounded(&full[s], (uint32_t)((j / C::S) & 1));
        ok = group_and(bar, C::GT, ok);
        if (!ok) {
            if (gt == 0) record_timeout(p.status);
            break;
        }
        char *slot = smem + s * C::SLOT_BYTES;
        if constexpr (H == W) ring_square<H, DIR, LAMF>(slot, gt, bar, p.sc, lam_s, p.lam);  // both end with a group barrier
        else ring_rect<H, W, DIR, LAMF>(slot, gt, bar, p.sc, p.lam);
        fence_proxy_async_smem();  // the TMA store reads the slot through the async proxy
        group_sync(bar, C::GT);
        if (gt == 0) mbar_arrive(&done[s]);
    }
}

// ---------------------------------------------------------------- host side
template <int H, int W, int DIR, bool LAMF = false>
static cudaError_t ring_launch_one(const DirScales &sc, const ExecGeom &g, unsigned int *status,
                                   cudaStream_t stream)
{
    using C = RingCfg<H, W, DIR>;
    auto kern = k_ring<H, W, DIR, LAMF>;
    static DeviceLaunchCache cache;
    int dev = 0, bps_dev = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cache.get(
        dev,
        [&](int d, int &bps, int &sms) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
            if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, C::THREADS, C::SMEM);
            if (r == cudaSuccess && bps < 1) r = cudaErrorInvalidConfiguration;
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
            if (r == cudaSuccess && debug_enabled())
                fprintf(stderr, "[bdct] k_ring<%d,%d,%d>: %d slots of %d B, %d groups x %d warps + producer, smem %zu B\n",
                        H, W, DIR, C::S, C::SLOT_BYTES, C::NG, C::GW, C::SMEM);
            return r;
        },
        &bps_dev, &num_sms);
    if (e != cudaSuccess) return e;
    (void)bps_dev;
    if (g.count <= 0) return cudaSuccess;
    RingParams p{};
    p.in = g.in;
    p.out = g.out;
    p.count = g.count;
    p.tiled = g.tiled;
    p.tiles_per_row = g.tiles_per_row;
    p.ld_in = g.ld_in;
    p.ld_out = g.ld_out;
    p.sc = sc;
    p.status = status;
    p.in_off = g.in_off;
    p.out_off = g.out_off;
    p.lam = g.lam;
    if ((DIR == DIR_SPEC || LAMF) && !g.lam) return cudaErrorInvalidValue;
    p.indexed = (g.in_off != nullptr || g.out_off != nullptr) ? 1 : 0;
    if (p.indexed) {
        if (!g.in_off || !g.out_off) return cudaErrorInvalidValue;
    } else if (g.tiled) {
        const unsigned long long rows = (unsigned long long)(g.count / g.tiles_per_row) * H;
        const unsigned long long cols = (unsigned long long)g.tiles_per_row * W;
        e = tma_map_2d(&p.map_in, g.in, rows, cols, (unsigned long long)g.ld_in, H);
        if (e == cudaSuccess) e = tma_map_2d(&p.map_out, g.out, rows, cols, (unsigned long long)g.ld_out, H);
        if (e != cudaSuccess) return e;
    } else {
        const unsigned long long rows = (unsigned long long)g.count * H;
        e = tma_map_2d(&p.map_in, g.in, rows, W, W, H);
        if (e == cudaSuccess) e = tma_map_2d(&p.map_out, g.out, rows, W, W, H);
        if (e != cudaSuccess) return e;
    }
    long long grid = num_sms;
    if (grid > g.count) grid = g.count;
    if ((g.count + grid - 1) / grid > 0x7fffff00LL) return cudaErrorInvalidValue;
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

template <int H, int W>
static cudaError_t ring_dir(Dir dir, const DirScales &sc, const ExecGeom &g, unsigned int *st, cudaStream_t s)
{
    switch (dir) {
        case DIR_FWD: return ring_launch_one<H, W, DIR_FWD>(sc, g, st, s);
        case DIR_INV: return ring_launch_one<H, W, DIR_INV>(sc, g, st, s);
        case DIR_SPEC:
            if constexpr (H == 64 && W == 64) return ring_launch_one<H, W, DIR_SPEC>(sc, g, st, s);
            else return cudaErrorInvalidValue;  // composed by the caller
        default: return ring_launch_one<H, W, DIR_RT>(sc, g, st, s);
    }
}

cudaError_t ring_forward_lam(int rows, int cols, const DirScales &sc, const ExecGeom &g, unsigned int *status,
                             cudaStream_t stream)
{
    if (rows == 64 && cols == 128) return ring_launch_one<64, 128, DIR_FWD, true>(sc, g, status, stream);
    if (rows == 128 && cols == 64) return ring_launch_one<128, 64, DIR_FWD, true>(sc, g, status, stream);
    if (rows == 128 && cols == 128) return ring_launch_one<128, 128, DIR_FWD, true>(sc, g, status, stream);
    return cudaErrorInvalidValue;
}

cudaError_t ring_launch(int rows, int cols, Dir dir, const DirScales &sc, const ExecGeom &g, unsigned int *status,
                        cudaStream_t stream)
{
    if (rows == 64 && cols == 64) return ring_dir<64, 64>(dir, sc, g, status, stream);
    if (rows == 64 && cols == 128) return ring_dir<64, 128>(dir, sc, g, status, stream);
    if (rows == 128 && cols == 64) return ring_dir<128, 64>(dir, sc, g, status, stream);
    if (rows == 128 && cols == 128) return ring_dir<128, 128>(dir, sc, g, status, stream);
    return cudaErrorInvalidValue;
}

}  // namespace bdct
