// FP32 fused 2D DCT kernels for small power-of-two sides (8, 16, 32, in
// every combination); sides 64 and 128 go to the ring kernels of
// fp32_ring.cu through the same entry points.
//
// What is computed: Eq. 2 of the BRiDCT paper, C(X) = Q_h X Q_w^T (forward,
// DCT-II), C^{-1}(Y) = Q_h^T Y Q_w (inverse, DCT-III) and the round trip,
// with Q_n = D_n G_n as in Eq. 3: G_n is the unscaled cosine kernel
// G[k][j] = cos(pi (2j+1) k / (2n)) and D_n the diagonal of Eq. 1.  The
// diagonal scales are folded into the pass outputs (forward), the pass inputs
// (inverse) or between the core and its adjoint (round trip, Prop. 1).
//
// 1D cores: dct_cores.cuh (even/odd DCT-II recursion, FFT-based DCT-IV).
//
// On-chip organization (the GPU counterpart of the paper's Algorithm 1 and of
// its Section 3.2 padded stride): arrays are staged in shared memory by TMA
// bulk copies, one array per 16-byte-padded slot; pass 1 gives each thread one
// column (or two adjacent columns), pass 2 one row (or two rows), and each
// line lives in registers while its 1D core runs; two lines of a thread run
// as one packed line (float2 cores: one packed FP32 instruction serves both).
// HBM traffic is one read and one write of every element.
#include <cuda_runtime.h>

#include "bdct_internal.h"
#include "dct_cores.cuh"
#include "ptx.cuh"

#include <cstdio>

namespace bdct {

// ------------------------------------------------------------ kernel
// Pipeline organization.  A persistent CTA of NW warps owns a ring of STAGES
// shared-memory stages; each stage holds a chunk of G arrays (or G adjacent
// image tiles).  Warp 0 fills stages ahead with TMA bulk copies completing on
// the stage's mbarrier and drains finished stages with TMA bulk stores, so
// HBM reads, the arithmetic and HBM writes of different chunks overlap; all
// warps share the arithmetic of a chunk.  Every thread waits on the stage's
// mbarrier itself; the CTA-wide agreement on that (bounded) wait comes at the
// barrier after pass 1, so warp 0's copy issue for the previous chunk does
// not hold the other warps back.
//
// Two shared-memory layouts, both bank-conflict-free for the column pass
// (one column per thread, scalar loads, or a column pair, 8-byte loads) and
// the row pass (one row per thread, 16-byte loads):
//  * contiguous batch -> "slots": array a at a*P, P = h*w + 4 floats, one bulk
//    copy per array; a warp instruction touches 8 arrays at once (4 adjacent
//    columns each in pass 1, one row each in pass 2), and the 16-byte gap
//    between slots spreads them over all 32 banks;
//  * tiled image -> "strip": the G tiles of a block row side by side, row r
//    at r*SP, SP = G*w + 4 floats, one bulk copy per image row; pass 1 lanes
//    take 32 adjacent strip columns (or column pairs), pass 2 lanes take 8
//    rows of one tile, which the odd 16-byte row pitch spreads over all banks.
// Shared-memory layouts of a stage (see the comment above).
enum Layout { LAY_SLOT = 0, LAY_STRIP = 1 };

template <int H, int W, bool TILED>
struct FusedCfg {
    static constexpr int HW = H * W;
    static constexpr int LAYOUT = TILED ? LAY_STRIP : LAY_SLOT;
    // arrays per chunk: contiguous batches of 256-element arrays take 16
    // (measured 0.82 -> 0.94 of HBM for 16 x 16); image strips of tiles at
    // most 16 wide and 256 elements take 16 (16-wide tiles: a column pair per
    // thread in pass 1; 16 x 8 tiles on a 4096^2 image 0.60 -> 0.81 of HBM,
    // 32 x 8 0.58 -> 0.63 against 8 tiles, whose CTAs had two warps), 32 x 16
    // tiles stay at 8 (no better with 16)
    static constexpr int G = (HW <= 64 || (LAYOUT == LAY_SLOT && HW == 256)) ? 16
                             : (LAYOUT == LAY_STRIP && W <= 16 && HW <= 256 ? 16 : 8);
    // pass 1 on two adjacent columns per thread (8-byte loads), run as one
    // packed line (float2 cores).  Pairing halves the warps of a CTA; measured
    // on contiguous batches it pays for 32 x 32 only (other shapes lose more
    // latency hiding than the packed instructions save)
    static constexpr bool PAIR1 = LAYOUT == LAY_STRIP ? W >= 16 : (H == 32 && W == 32);
    // warps: every thread has at least one line (or column pair) in each pass
    static constexpr int NW_P1 = G * W / (PAIR1 ? 64 : 32);
    static constexpr int NW_P2 = G * H / 32;
    static constexpr int NW_MAX = NW_P1 < NW_P2 ? NW_P1 : NW_P2;
    static constexpr int NW = NW_MAX > 8 ? 8 : NW_MAX;  // warps per CTA
    static constexpr int THREADS = 32 * NW;
    static constexpr int P = HW + 4;       // slot pitch (floats)
    static constexpr int SP = G * W + 4;   // strip row pitch (floats)
    static constexpr int STAGE_FLOATS =
        LAYOUT == LAY_STRIP ? H * SP : G * P;
    static constexpr int STAGE_BYTES = STAGE_FLOATS * 4;
    static constexpr int ST_RAW = (32 * 1024) / STAGE_BYTES;
    static constexpr int STAGES = ST_RAW < 2 ? 2 : (ST_RAW > 4 ? 4 : ST_RAW);
    static constexpr int J1 = G * W / (PAIR1 ? 2 * THREADS : THREADS);  // column steps per thread (pass 1)
    static constexpr int J2 = G * H / THREADS;  // rows per thread (pass 2)
    // pass 2 rows in packed pairs (line_op2) when a thread has an even number
    // of rows; measured, it pays on image strips (the 16 x 16 image step runs
    // 10% faster) and is mixed on contiguous batches
    static constexpr bool PAIR2 = LAYOUT == LAY_STRIP && J2 % 2 == 0 && W >= 4;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + STAGES * 8;
    // spectral direction: the folded diagonal staged once per CTA, rows at a
    // pitch of W + 4 floats (the eight rows a row-pass instruction touches
    // fall on distinct banks)
    static constexpr int LAM_P = W + 4;
    static constexpr size_t LAM_BYTES = (size_t)H * LAM_P * 4 + 8;  // + the alignment pad
    // register-allocation hint (resident CTAs per SM; 0 = none).  Measured: the
    // image strips and the 64-element batches run faster with the allocation
    // the hint gives (16x16 image step 15.0 -> 14.65 us, 8x8 round trip 0.76
    // -> 0.80 of HBM), the other batches without it (16x16 0.93 -> 0.86 with)
    static constexpr int MIN_CTAS = TILED ? 2 : (HW <= 64 ? 1 : 0);
    static_assert(J1 >= 1 && J2 >= 1 && J1 * THREADS * (PAIR1 ? 2 : 1) == G * W && J2 * THREADS == G * H,
                  "lane mapping");
    static_assert((P % 8) == 4 && (SP % 8) == 4, "pitches must be 4 mod 8 floats");
    static_assert(LAYOUT == LAY_STRIP || G % 8 == 0, "slot-layout lanes span 8 arrays");
    static_assert(H <= 32 && W <= 32, "sides 64 and 128 use the ring kernels");
};

// Element (a, r, c) of a stage: array/tile a, row r, column c.
template <int H, int W, bool TILED>
__device__ __forceinline__ int elem(int a, int r, int c)
{
    using C = FusedCfg<H, W, TILED>;
    if constexpr (C::LAYOUT == LAY_STRIP) return r * C::SP + a * W + c;
    else return a * C::P + r * W + c;
}

// Row stride of a stage in floats.
template <int H, int W, bool TILED>
__device__ __forceinline__ constexpr int row_stride()
{
    using C = FusedCfg<H, W, TILED>;
    return C::LAYOUT == LAY_STRIP ? C::SP : W;
}

// Pass 1 line j of this thread -> (array, column).
template <int H, int W, bool TILED>
__device__ __forceinline__ void map_col(int j, int warp, int lane, int &a, int &col)
{
    using C = FusedCfg<H, W, TILED>;
    if constexpr (C::LAYOUT == LAY_SLOT) {
        const int combo = warp + C::NW * j;
        a = (lane & 7) + 8 * (combo % (C::G / 8));
        col = (lane >> 3) + 4 * (combo / (C::G / 8));
    } else {
        // 32 adjacent columns of the strip
        const int s = lane + 32 * (warp + C::NW * j);
        a = s / W;
        col = s % W;
    }
}

// Pass 2 line j of this thread -> (array, row).
template <int H, int W, bool TILED>
__device__ __forceinline__ void map_row(int j, int warp, int lane, int &a, int &r)
{
    using C = FusedCfg<H, W, TILED>;
    if constexpr (C::LAYOUT == LAY_SLOT) {
        const int combo = warp + C::NW * j;
        a = (lane & 7) + 8 * (combo % (C::G / 8));
        r = (lane >> 3) + 4 * (combo / (C::G / 8));
    } else {
        const int u = (lane >> 3) + 4 * (warp + C::NW * j);
        a = u % C::G;
        r = (lane & 7) + 8 * (u / C::G);
    }
}

struct FusedParams {
    const float *in;
    float *out;
    long long count;      // arrays (contiguous) or tiles (tiled)
    int tiles_per_row;    // tiled only
    int chunks_per_row;   // tiled only: ceil(tiles_per_row / G)
    long long ld_in, ld_out;  // tiled only (floats)
    int nchunks;          // < 2^31, checked by the host
    DirScales sc;
    unsigned int *status;
    const long long *in_off, *out_off;  // indexed batch, or null
    const float *lam;     // spectral only: folded diagonal, h x w
};

// Start of array a of the batch (contiguous or indexed).
__device__ __forceinline__ const float *arr_in(const FusedParams &p, long long a, int hw)
{
    return p.in_off ? p.in + p.in_off[a] : p.in + a * hw;
}
__device__ __forceinline__ float *arr_out(const FusedParams &p, long long a, int hw)
{
    return p.out_off ? p.out + p.out_off[a] : p.out + a * hw;
}

// Where a chunk lives: arrays [first, first + n) of a contiguous batch, or
// tiles t0 .. t0 + n - 1 of block row brow of an image.
struct ChunkGeom {
    long long first;
    long long brow;
    int n, t0;
};

template <int H, int W, bool TILED>
__device__ __forceinline__ ChunkGeom chunk_geom(const FusedParams &p, int c)
{
    using C = FusedCfg<H, W, TILED>;
    ChunkGeom g;
    if constexpr (!TILED) {
        g.first = (long long)c * C::G;
        const long long rem = p.count - g.first;
        g.n = rem < C::G ? (int)rem : C::G;
        g.brow = 0;
        g.t0 = 0;
    } else {
        const unsigned int br = (unsigned int)c / (unsigned int)p.chunks_per_row;
        g.brow = br;
        g.t0 = (int)((unsigned int)c - br * (unsigned int)p.chunks_per_row) * C::G;
        const int rem = p.tiles_per_row - g.t0;
        g.n = rem < C::G ? rem : C::G;
        g.first = 0;
    }
    return g;
}

// Issue the copies that fill one stage (all lanes of warp 0).
template <int H, int W, bool TILED>
__device__ __forceinline__ void issue_fill(const FusedParams &p, const ChunkGeom &g, float *stage, uint64_t *bar,
                                           int lane)
{
    using C = FusedCfg<H, W, TILED>;
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(g.n * C::HW * 4));
    __syncwarp();
    if constexpr (C::LAYOUT == LAY_SLOT) {
        for (int a = lane; a < g.n; a += 32)
            bulk_load(stage + a * C::P, arr_in(p, g.first + a, C::HW), C::HW * 4, bar);
    } else {
        for (int r = lane; r < H; r += 32) {
            const float *src = p.in + (g.brow * H + r) * p.ld_in + (long long)g.t0 * W;
            bulk_load(stage + r * C::SP, src, (uint32_t)(g.n * W * 4), bar);
        }
    }
}

// Issue the copies that drain one stage (all lanes of warp 0).
template <int H, int W, bool TILED>
__device__ __forceinline__ void issue_drain(const FusedParams &p, const ChunkGeom &g, const float *stage, int lane)
{
    using C = FusedCfg<H, W, TILED>;
    if constexpr (C::LAYOUT == LAY_SLOT) {
        for (int a = lane; a < g.n; a += 32) bulk_store(arr_out(p, g.first + a, C::HW), stage + a * C::P, C::HW * 4);
    } else {
        for (int r = lane; r < H; r += 32) {
            float *dst = p.out + (g.brow * H + r) * p.ld_out + (long long)g.t0 * W;
            bulk_store(dst, stage + r * C::SP, (uint32_t)(g.n * W * 4));
        }
    }
}

// Error path: the copies issued for chunks first .. filled - 1 of this CTA
// (chunk i in stage i mod stages, phase (i / stages) mod 2) land, each wait
// bounded, before the CTA exits.
__device__ __forceinline__ void drain_fills(uint64_t *full, int stages, int first, int filled)
{
    for (int i = first; i < filled; ++i)
        if (!mbar_wait_bounded(&full[i % stages], (uint32_t)((i / stages) & 1))) break;
}

template <int NW>
__device__ __forceinline__ void cta_sync()
{
    if constexpr (NW == 1) __syncwarp();
    else __syncthreads();
}

// Column pass over one stage: one column (or two adjacent columns, as one
// packed line) per thread per step, 1D operation OP along h (a direction of
// line_op, or an unscaled core).
template <int H, int W, bool TILED, int OP>
__device__ __forceinline__ void col_pass(float *stage, int n, int warp, int lane, AxisScale sc)
{
    using C = FusedCfg<H, W, TILED>;
    if constexpr (C::PAIR1) {
#pragma unroll
        for (int j = 0; j < C::J1; ++j) {
            int a, col;
            if constexpr (C::LAYOUT == LAY_STRIP) {
                const int s2 = 2 * (lane + 32 * (warp + C::NW * j));  // even strip column
                a = s2 / W;
                col = s2 % W;
            } else {
                // lanes: 8 arrays x 4 column pairs; with the 4-mod-8 slot pitch each
                // half-warp's 8-byte accesses cover the 32 banks once
                const int combo = warp + C::NW * j;
                a = (lane & 7) + 8 * (combo % (C::G / 8));
                col = 2 * ((lane >> 3) + 4 * (combo / (C::G / 8)));
            }
            if (a < n) {
                // the two columns run as one packed line (float2 cores)
                float2 *q = reinterpret_cast<float2 *>(stage + elem<H, W, TILED>(a, 0, col));
                constexpr int RS2 = row_stride<H, W, TILED>() / 2;
                float2 x[H];
#pragma unroll
                for (int i = 0; i < H; ++i) x[i] = q[i * RS2];
                line_op<H, OP, float2>(x, sc);
#pragma unroll
                for (int i = 0; i < H; ++i) q[i * RS2] = x[i];
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < C::J1; ++j) {
            int a, col;
            map_col<H, W, TILED>(j, warp, lane, a, col);
            if (a < n) {
                float *q = stage + elem<H, W, TILED>(a, 0, col);
                constexpr int RS = row_stride<H, W, TILED>();
                float x[H];
#pragma unroll
                for (int i = 0; i < H; ++i) x[i] = q[i * RS];
                line_op<H, OP>(x, sc);
#pragma unroll
                for (int i = 0; i < H; ++i) q[i * RS] = x[i];
            }
        }
    }
}

// Row pass over one stage: one row per thread per step, 1D operation along w;
// with an even number of rows per thread the rows go in packed pairs.  For
// the spectral direction each row k runs transform -- row k of the folded
// diagonal -- adjoint (line_spectral).
template <int H, int W, bool TILED, int DIR>
__device__ __forceinline__ void row_pass(float *stage, int n, int warp, int lane, AxisScale sc, const float *lam)
{
    using C = FusedCfg<H, W, TILED>;
    // row r of the spectrum after the column pass holds frequency r along h;
    // lam: the folded diagonal in shared memory, pitch LAM_P
    auto lam_row = [&](int r, float (&d)[W]) {
        const float4 *lr = reinterpret_cast<const float4 *>(lam + r * C::LAM_P);
#pragma unroll
        for (int v = 0; v < W / 4; ++v) {
            const float4 t = lr[v];
            d[4 * v] = t.x; d[4 * v + 1] = t.y; d[4 * v + 2] = t.z; d[4 * v + 3] = t.w;
        }
    };
    if constexpr (C::PAIR2) {
#pragma unroll
        for (int j = 0; j < C::J2; j += 2) {
            int a0, r0, a1, r1;
            map_row<H, W, TILED>(j, warp, lane, a0, r0);
            map_row<H, W, TILED>(j + 1, warp, lane, a1, r1);
            const bool v0 = a0 < n, v1 = a1 < n;
            float4 *q0 = reinterpret_cast<float4 *>(stage + elem<H, W, TILED>(v0 ? a0 : 0, r0, 0));
            float4 *q1 = reinterpret_cast<float4 *>(stage + elem<H, W, TILED>(v1 ? a1 : 0, r1, 0));
            float x0[W], x1[W];
#pragma unroll
            for (int v = 0; v < W / 4; ++v) {
                const float4 t0 = q0[v], t1 = q1[v];
                x0[4 * v] = t0.x; x0[4 * v + 1] = t0.y; x0[4 * v + 2] = t0.z; x0[4 * v + 3] = t0.w;
                x1[4 * v] = t1.x; x1[4 * v + 1] = t1.y; x1[4 * v + 2] = t1.z; x1[4 * v + 3] = t1.w;
            }
            if constexpr (DIR == DIR_SPEC) {
                float d0[W], d1[W];
                lam_row(r0, d0);
                lam_row(r1, d1);
                line_spectral2<W>(x0, x1, d0, d1);
            } else {
                line_op2<W, DIR>(x0, x1, sc);
            }
            if (v0) {
#pragma unroll
                for (int v = 0; v < W / 4; ++v) q0[v] = make_float4(x0[4 * v], x0[4 * v + 1], x0[4 * v + 2], x0[4 * v + 3]);
            }
            if (v1) {
#pragma unroll
                for (int v = 0; v < W / 4; ++v) q1[v] = make_float4(x1[4 * v], x1[4 * v + 1], x1[4 * v + 2], x1[4 * v + 3]);
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < C::J2; ++j) {
            int a, r;
            map_row<H, W, TILED>(j, warp, lane, a, r);
            if (a < n) {
                float4 *q = reinterpret_cast<float4 *>(stage + elem<H, W, TILED>(a, r, 0));
                float x[W];
#pragma unroll
                for (int v = 0; v < W / 4; ++v) {
                    const float4 t = q[v];
                    x[4 * v] = t.x; x[4 * v + 1] = t.y; x[4 * v + 2] = t.z; x[4 * v + 3] = t.w;
                }
                if constexpr (DIR == DIR_SPEC) {
                    float d[W];
                    lam_row(r, d);
                    line_spectral<W>(x, d);
                } else {
                    line_op<W, DIR>(x, sc);
                }
#pragma unroll
                for (int v = 0; v < W / 4; ++v) q[v] = make_float4(x[4 * v], x[4 * v + 1], x[4 * v + 2], x[4 * v + 3]);
            }
        }
    }
}

// One wave of 16 x 16 image strips: every chunk gets a CTA of its own, seven
// CTAs per SM (at most 73 registers; the launch pads the shared memory so
// that no eighth CTA lands on an SM; with the two-stage ring six CTAs fit,
// and a 2048^2 image's 1024 chunks left 112 CTAs a second chunk).  Warp w
// owns tiles 4w .. 4w + 3 of the chunk in both passes -- strip columns
// 64w .. 64w + 63: pass 1 gives each lane one column pair, pass 2 rows r and
// r + 8 of one of the four tiles -- so each warp loads, transforms and
// stores its quarter on an mbarrier of its own and never waits for the rest
// of the chunk.  Measured on a 2048^2 image: 8.59 us per inverse launch with
// the two-stage ring, 8.26 with one wave of whole-chunk CTAs, 7.57 with
// warp-owned quarters (14.65 -> 14.0 -> 12.98 us per forward-then-inverse
// step).
constexpr int kOneWaveCtas = 7;

// Named barrier 1 over `nthreads` threads that also ANDs v over them.
__device__ __forceinline__ bool part_sync_and(bool v, int nthreads)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(nthreads)
        : "memory");
    return r != 0;
}

template <int DIR>
__global__ void __launch_bounds__(FusedCfg<16, 16, true>::THREADS, kOneWaveCtas) k_strip16_wave(const FusedParams p)
{
    constexpr int H = 16, W = 16;
    using C = FusedCfg<H, W, true>;
    static_assert(C::PAIR1 && C::J1 == 1 && C::J2 == 2 && C::NW * 4 == C::G, "warp-owned quarters");
    extern __shared__ __align__(128) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + C::STAGE_FLOATS) + warp;
    // spectral only: the folded diagonal, after the warps' barriers
    float *lam_s = reinterpret_cast<float *>(smem + C::STAGE_FLOATS) + 2 * C::NW;
    const ChunkGeom g = chunk_geom<H, W, true>(p, (int)blockIdx.x);
    int nq = g.n - 4 * warp;  // tiles of this warp
    nq = nq < 0 ? 0 : (nq > 4 ? 4 : nq);
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    pdl_launch_dependents();
    pdl_wait_prerequisites();
    if constexpr (DIR == DIR_SPEC) {
        for (int e = threadIdx.x; e < H * W; e += C::THREADS) lam_s[(e / W) * C::LAM_P + e % W] = __ldg(p.lam + e);
        __syncthreads();
    }
    if (nq == 0) return;
    float *qs = smem + 64 * warp;  // the warp's columns of strip row 0
    const long long c0 = (long long)(g.t0 + 4 * warp) * W;
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(nq * H * W * 4));
    __syncwarp();
    if (lane < H) bulk_load(qs + lane * C::SP, p.in + (g.brow * H + lane) * p.ld_in + c0, (uint32_t)(nq * W * 4), bar);
    if constexpr (DIR == DIR_SPEC) {
        // the chunk is stored from warp 0 as in the inverse below; a warp
        // whose wait expired still arrives at the barrier (with false), so
        // that nothing is stored and no warp is left waiting
        // (the barrier's thread count is recomputed where it is used: held
        // across the passes it took a register, and this form sits at the
        // 72-register ceiling)
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, 0))) {
            if (lane == 0) {
                record_timeout(p.status);
                mbar_wait_bounded(bar, 0);
            }
            part_sync_and(false, 32 * ((g.n + 3) / 4));
            return;
        }
        col_pass<H, W, true, CORE_FWD>(smem, g.n, warp, lane, p.sc.h);
        __syncwarp();
        row_pass<H, W, true, DIR>(smem, g.n, warp, lane, p.sc.w, lam_s);
        __syncwarp();
        col_pass<H, W, true, CORE_INV>(smem, g.n, warp, lane, p.sc.h);
        fence_proxy_async_smem();
        if (part_sync_and(true, 32 * ((g.n + 3) / 4)) && warp == 0 && lane < H) {
            bulk_store(p.out + (g.brow * H + lane) * p.ld_out + (long long)g.t0 * W, smem + lane * C::SP,
                       (uint32_t)(g.n * W * 4));
            bulk_commit();
            bulk_wait<0>();
        }
    } else if constexpr (DIR == DIR_FWD) {
        // each warp stores its own quarter
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, 0))) {
            // nothing is stored; the copies land (bounded wait) before the exit
            if (lane == 0) {
                record_timeout(p.status);
                mbar_wait_bounded(bar, 0);
            }
            return;
        }
        col_pass<H, W, true, DIR>(smem, g.n, warp, lane, p.sc.h);
        __syncwarp();
        row_pass<H, W, true, DIR>(smem, g.n, warp, lane, p.sc.w, lam_s);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane < H) {
            bulk_store(p.out + (g.brow * H + lane) * p.ld_out + c0, qs + lane * C::SP, (uint32_t)(nq * W * 4));
            bulk_commit();
            bulk_wait<0>();
        }
    } else {
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, 0));
        if (!ok && lane == 0) {
            // nothing is stored; this quarter's copies land (bounded wait)
            record_timeout(p.status);
            mbar_wait_bounded(bar, 0);
        }
        if (ok) {
            col_pass<H, W, true, DIR>(smem, g.n, warp, lane, p.sc.h);
            __syncwarp();
            row_pass<H, W, true, DIR>(smem, g.n, warp, lane, p.sc.w, lam_s);
            fence_proxy_async_smem();
        }
        // The inverse and the round trip store the whole chunk from warp 0, in
        // whole 1 KiB rows, once every warp with tiles is done (named barrier
        // 1 over those warps, which also ANDs their outcomes: a warp whose
        // wait expired still arrives, and then nothing is stored).  Measured
        // on a 2048^2 image: inverse 7.50 -> 7.40 us per launch, round trip
        // 8.24 -> 8.02, the spectral form above 9.40 -> 9.14; the forward
        // keeps its per-warp stores (7.38 us either way).  The spectral form
        // sits at the 72-register ceiling of seven CTAs per SM and keeps an
        // early exit for its passes: with the passes made conditional on the
        // wait outcome instead, it spilled and ran at half speed.
        if (part_sync_and(ok, 32 * ((g.n + 3) / 4)) && warp == 0 && lane < H) {
            bulk_store(p.out + (g.brow * H + lane) * p.ld_out + (long long)g.t0 * W, smem + lane * C::SP,
                       (uint32_t)(g.n * W * 4));
            bulk_commit();
            bulk_wait<0>();
        }
    }
}

template <int H, int W, int DIR, bool TILED>
__global__ void __launch_bounds__(FusedCfg<H, W, TILED>::THREADS, FusedCfg<H, W, TILED>::MIN_CTAS)
    k_fused(const FusedParams p)
{
    using C = FusedCfg<H, W, TILED>;
    constexpr int STAGES = C::STAGES;
    extern __shared__ __align__(128) float smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * C::STAGE_FLOATS);
    // spectral only: the folded diagonal, 16-byte aligned after the barriers
    float *lam_s = reinterpret_cast<float *>(full + ((STAGES + 1) & ~1));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grid = (int)gridDim.x;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    // the next kernel may start launching; global memory is touched only
    // after every prerequisite grid has finished
    pdl_launch_dependents();
    pdl_wait_prerequisites();
    if constexpr (DIR == DIR_SPEC) {
        for (int e = tid; e < H * W; e += C::THREADS) lam_s[(e / W) * C::LAM_P + e % W] = __ldg(p.lam + e);
    }
    __syncthreads();

    // prologue: fill every stage (chunk k of this CTA uses stage k mod STAGES,
    // phase (k / STAGES) mod 2)
    if (warp == 0) {
        for (int s = 0; s < STAGES; ++s) {
            const int c = (int)blockIdx.x + s * grid;
            if (c < p.nchunks)
                issue_fill<H, W, TILED>(p, chunk_geom<H, W, TILED>(p, c), smem + s * C::STAGE_FLOATS, &full[s], lane);
        }
    }
    // refill policy (see the end of the loop): the round trip and the spectral
    // direction carry twice the arithmetic of one direction
    constexpr bool DEFER = STAGES >= 3 || (STAGES == 2 && DIR != DIR_RT && DIR != DIR_SPEC);

    int failed_at = -1;   // iteration whose stage wait expired, if any
    int s = 0;            // stage of the current chunk
    uint32_t phase = 0;   // parity of the stage's current use
    int prev_s = 0;
    for (int c = (int)blockIdx.x, k = 0; c < p.nchunks; c += grid, ++k) {
        float *stage = smem + s * C::STAGE_FLOATS;
        // each thread waits for the stage itself; the CTA agrees on the outcome
        // at the barrier after pass 1, so that the other warps start a chunk
        // while warp 0 still issues the copies of the previous one (pass 1 on a
        // stage whose wait expired only wastes work: nothing is stored)
        bool ok = mbar_wait_bounded(&full[s], phase);
        const ChunkGeom g = chunk_geom<H, W, TILED>(p, c);
        const int n = g.n;

        // pass 1: columns, 1D operation along h (the spectral direction runs
        // the unscaled forward core; its scales live in the folded diagonal)
        col_pass<H, W, TILED, DIR == DIR_SPEC ? CORE_FWD : DIR>(stage, n, warp, lane, p.sc.h);
        if constexpr (C::NW == 1) ok = __all_sync(0xffffffffu, ok);
        else ok = __syncthreads_and(ok);
        if (!ok) {
            failed_at = k;
            break;
        }

        // pass 2: rows, 1D operation along w
        row_pass<H, W, TILED, DIR>(stage, n, warp, lane, p.sc.w, lam_s);
        if constexpr (DIR == DIR_SPEC) {
            // pass 3 (spectral only): columns, unscaled adjoint core along h
            cta_sync<C::NW>();
            col_pass<H, W, TILED, CORE_INV>(stage, n, warp, lane, p.sc.h);
        }
        fence_proxy_async_smem();
        cta_sync<C::NW>();

        if (warp == 0) {
            // bulk groups are per thread: every lane commits the stores it issued
            issue_drain<H, W, TILED>(p, g, stage, lane);
            bulk_commit();
            // Deferred refill: the stage drained in the previous iteration, once its
            // reads are done (no wait on the stores just issued).  With two stages
            // that loads the next chunk only now; the round trip (twice the
            // arithmetic per chunk) instead refills this stage right away, which
            // measured 0.81 -> 0.94 of HBM on 32 x 32 batches, while forward and
            // inverse lose more to the wait on the stores than they gain.
            if constexpr (DEFER) {
                if (k >= 1) {
                    const int cn = c + (STAGES - 1) * grid;
                    if (cn < p.nchunks) {
                        bulk_wait_read<1>();
                        __syncwarp();
                        issue_fill<H, W, TILED>(p, chunk_geom<H, W, TILED>(p, cn), smem + prev_s * C::STAGE_FLOATS,
                                                &full[prev_s], lane);
                    }
                }
            } else {
                // refill this stage as soon as its stores have read it, so that the
                // chunk after next loads while the next is transformed
                const int cn = c + STAGES * grid;
                if (cn < p.nchunks) {
                    bulk_wait_read<0>();
                    __syncwarp();
                    issue_fill<H, W, TILED>(p, chunk_geom<H, W, TILED>(p, cn), stage, &full[s], lane);
                }
            }
        }
        prev_s = s;
        if (++s == STAGES) { s = 0; phase ^= 1u; }
    }
    if (failed_at >= 0 && tid == 0) {
        record_timeout(p.status);
        // chunks whose copies were issued by then: the prologue's, plus one
        // refill per finished iteration (from the second on when deferred)
        const int k = failed_at;
        const int n_own = (p.nchunks - (int)blockIdx.x + grid - 1) / grid;
        int issued = DEFER ? (k + STAGES - 1 > STAGES ? k + STAGES - 1 : STAGES) : k + STAGES;
        if (issued > n_own) issued = n_own;
        drain_fills(full, STAGES, k, issued);
    }
    if (warp == 0) bulk_wait<0>();
}

// ------------------------------------------------------------ host side
__global__ void k_gen_cos_table(float *t)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > 4096) return;
    // cos(pi r / 8192) in FP64 with an exact argument; exact 0 at r = 4096.
    t[r] = (r == 4096) ? 0.0f : (float)cospi((double)r / 8192.0);
}

__global__ void k_gen_cos_table3(float *t)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > 768) return;
    // cos(pi r / 1536) in FP64; exact 0 at r = 768
    t[r] = (r == 768) ? 0.0f : (float)cospi((double)r / 1536.0);
}

static std::mutex g_table_mutex;
static bool g_table_ready[64];

cudaError_t fused_init_device(int device)
{
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_table_mutex);
    if (g_table_ready[device]) return cudaSuccess;
    float *tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, 4097 * sizeof(float));
    if (e != cudaSuccess) return e;
    k_gen_cos_table<<<(4097 + 255) / 256, 256>>>(tmp);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = init_cos_table(tmp);
    if (e == cudaSuccess) e = lines_init_table(tmp);
    if (e == cudaSuccess) e = ring_init_table(tmp);
    if (e == cudaSuccess) {
        k_gen_cos_table3<<<(769 + 255) / 256, 256>>>(tmp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = init_cos_table3(tmp);
    if (e == cudaSuccess) e = lines_init_table3(tmp);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(tmp);
    if (e == cudaSuccess) g_table_ready[device] = true;
    return e;
}

bool fused_supported(int rows, int cols)
{
    auto ok = [](int n) { return n == 8 || n == 16 || n == 32; };
    return (ok(rows) && ok(cols)) || ring_supported(rows, cols);
}

template <int H, int W, int DIR, bool TILED>
static cudaError_t launch_one(const DirScales &sc, const ExecGeom &g, unsigned int *status, cudaStream_t stream)
{
    using C = FusedCfg<H, W, TILED>;
    auto kern = k_fused<H, W, DIR, TILED>;
    constexpr size_t smem = C::SMEM + (DIR == DIR_SPEC ? C::LAM_BYTES : 0);
    static DeviceLaunchCache cache;
    int dev = 0, blocks_per_sm = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cache.get(
        dev,
        [&](int d, int &bps, int &sms) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, C::THREADS, smem);
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
            if (r == cudaSuccess && bps < 1) r = cudaErrorInvalidConfiguration;
            if (r == cudaSuccess && debug_enabled())
                fprintf(stderr, "[bdct] k_fused<%d,%d,%d,%d>: %d CTAs/SM x %d threads, %d stages, smem %zu B\n", H, W,
                        DIR, (int)TILED, bps, C::THREADS, C::STAGES, smem);
            return r;
        },
        &blocks_per_sm, &num_sms);
    if (e != cudaSuccess) return e;
    FusedParams p{};
    p.in = g.in;
    p.out = g.out;
    p.count = g.count;
    p.tiles_per_row = g.tiles_per_row;
    p.ld_in = g.ld_in;
    p.ld_out = g.ld_out;
    p.sc = sc;
    p.status = status;
    p.in_off = g.in_off;
    p.out_off = g.out_off;
    p.lam = g.lam;
    if (DIR == DIR_SPEC && !p.lam) return cudaErrorInvalidValue;
    long long nch;
    if (!TILED) {
        nch = (g.count + C::G - 1) / C::G;
    } else {
        p.chunks_per_row = (g.tiles_per_row + C::G - 1) / C::G;
        nch = (g.count / g.tiles_per_row) * p.chunks_per_row;
    }
    if (nch <= 0) return cudaSuccess;
    if (nch > 0x7ff00000LL) return cudaErrorInvalidValue;  // keeps c + STAGES * grid within int
    p.nchunks = (int)nch;
    // persistent: as many CTAs as fit on the device
    long long grid = (long long)blocks_per_sm * num_sms;
    if (grid > p.nchunks) grid = p.nchunks;
    auto launch_kern = kern;
    size_t launch_smem = smem;
    if constexpr (TILED && H == 16 && W == 16 && C::STAGES > 1) {
        // one CTA per chunk (k_strip16_wave) whenever all of them fit in one
        // wave of kOneWaveCtas per SM; the persistent ring for more
        auto kern1 = k_strip16_wave<DIR>;
        constexpr size_t need1 = (size_t)C::STAGE_BYTES + 8 * C::NW + (DIR == DIR_SPEC ? C::LAM_BYTES : 0);
        static DeviceLaunchCache cache1;
        static size_t smem1_dev[64];
        int bps1 = 0, sms1 = 0;
        e = cache1.get(
            dev,
            [&](int d, int &bps, int &sms) {
                // the shared memory of one of kOneWaveCtas CTAs (less the
                // 1 KiB the SM reserves per CTA), so that no more fit
                int per_sm = 0;
                cudaError_t r = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, d);
                size_t sm1 = need1;
                if (r == cudaSuccess) {
                    const size_t cap = ((size_t)per_sm / kOneWaveCtas - 1024) & ~(size_t)127;
                    if (cap > sm1) sm1 = cap;
                    smem1_dev[d] = sm1;
                }
                if (r == cudaSuccess) r = cudaFuncSetAttribute(kern1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
                if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern1, C::THREADS, sm1);
                if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
                if (r == cudaSuccess && debug_enabled())
                    fprintf(stderr, "[bdct] k_strip16_wave<%d>: %d CTAs/SM, smem %zu B\n", DIR, bps, sm1);
                return r;
            },
            &bps1, &sms1);
        if (e != cudaSuccess) return e;
        if (bps1 == kOneWaveCtas && (long long)p.nchunks <= (long long)bps1 * sms1) {
            launch_kern = kern1;
            launch_smem = smem1_dev[dev];
            grid = p.nchunks;
        }
    }
    // programmatic dependent launch: this grid may be scheduled while the
    // previous kernel in the stream drains; it waits for it before any access
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(C::THREADS);
    cfg.dynamicSmemBytes = launch_smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, launch_kern, p);
}

template <int H, int W>
static cudaError_t launch_hw(Dir dir, const DirScales &sc, const ExecGeom &g, unsigned int *st, cudaStream_t s)
{
    const bool t = g.tiled != 0;
    switch (dir) {
        case DIR_FWD: return t ? launch_one<H, W, DIR_FWD, true>(sc, g, st, s) : launch_one<H, W, DIR_FWD, false>(sc, g, st, s);
        case DIR_INV: return t ? launch_one<H, W, DIR_INV, true>(sc, g, st, s) : launch_one<H, W, DIR_INV, false>(sc, g, st, s);
        case DIR_RT: return t ? launch_one<H, W, DIR_RT, true>(sc, g, st, s) : launch_one<H, W, DIR_RT, false>(sc, g, st, s);
        default: return t ? launch_one<H, W, DIR_SPEC, true>(sc, g, st, s) : launch_one<H, W, DIR_SPEC, false>(sc, g, st, s);
    }
}

template <int H>
static cudaError_t launch_h(int cols, Dir dir, const DirScales &sc, const ExecGeom &g, unsigned int *st,
                            cudaStream_t s)
{
    switch (cols) {
        case 8: return launch_hw<H, 8>(dir, sc, g, st, s);
        case 16: return launch_hw<H, 16>(dir, sc, g, st, s);
        case 32: return launch_hw<H, 32>(dir, sc, g, st, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fused_launch(int rows, int cols, Dir dir, const DirScales &sc, const ExecGeom &g,
                         unsigned int *status, cudaStream_t stream)
{
    if (ring_supported(rows, cols)) {
        if (dir == DIR_SPEC) return cudaErrorInvalidValue;  // composed by the caller from F, scale, I
        return ring_launch(rows, cols, dir, sc, g, status, stream);
    }
    switch (rows) {
        case 8: return launch_h<8>(cols, dir, sc, g, status, stream);
        case 16: return launch_h<16>(cols, dir, sc, g, status, stream);
        case 32: return launch_h<32>(cols, dir, sc, g, status, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bdct
