// Split-BF16 tensor-core separable passes (tcgen05, FP32 accumulation in TMEM)
// for the shapes the on-chip tensor-core kernel (tc_split.cu, squares 16..64)
// does not hold: squares 128 and up, rectangles, whole large arrays, and the
// 8 x 8 blocks as one Kronecker product.
//
// What is computed: Eq. 2 of the BRiDCT paper, Y = M_h X M_w^T, as two
// passes of one contraction each.  A pass takes every row of every array
// (R rows of length K per array), applies the 1D operator M (N x K, the
// direction's matrix of Eq. 1 or of the REDFT pair) to it and writes the
// result transposed, out[b][n][r] = sum_k M[n][k] X[b][r][k]; two passes
// (rows, then the rows of the transposed intermediate) give the 2D transform
// in natural layout.  For 8 x 8 arrays one pass with the 64 x 64 Kronecker
// operator Q (x) Q over the vectorized array (R = 1) gives it directly.
// Direct matrix evaluation costs K multiply-adds per point (Section 1.2); the
// tensor cores take them.
//
// Exactness (Section 1.1 excludes approximated matrices): each FP32 input is
// split in the kernel into three BF16 terms x = x0 + x1 + x2 (each the
// round-to-nearest BF16 of the remaining residual), the FP64 operator into
// three terms once at plan time, and the six products with term orders
// summing to at most 2 are accumulated in FP32, smallest first.  Measured on
// the GPU, the tensor cores' FP32 accumulation loses about half an FP32 ulp
// per accumulated MMA step, always in the same direction, so one accumulator
// over a whole long contraction drifts linearly with its length (1.6e-6 at
// 1024 points, 7.7e-6 at 4096).  Each K chunk (at most 64 points, four MMA
// steps per product) therefore gets a fresh TMEM accumulator, and the
// threads add the chunk partials in registers with round-to-nearest FP32
// additions, in chunk order.

// Organization: a tile is 128 rows (the MMA's M) by NT <= 64 outputs (its N);
// K runs in chunks of KC <= 64 through two shared-memory stages and two TMEM
// accumulators.  All 128
// threads stage A -- thread t loads row t of the chunk (prefetched into
// registers one chunk ahead), splits it and writes the terms in the
// canonical K-major layout -- while thread 0 brings the operator's terms for
// the chunk with one bulk copy and, once both are in, issues the products
// and commits them to the stage's mbarrier.  The next chunk is staged while
// those products run, and the partial of chunk g - 2 is read from its TMEM
// lane (row t of the tile) into the running sums.  Epilogue: thread t stores
// its outputs transposed (lanes of a warp hold consecutive rows, so each
// output index is one coalesced segment).  Persistent CTAs walk the (row
// tile, output tile) items.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdio>

#include "bdct_internal.h"
#include "ptx.cuh"
#include "tc_ptx.cuh"

namespace bdct {

constexpr int kTgM = 128;     // rows per tile
constexpr int kTgKC = 64;     // largest K chunk
constexpr int kTgStages = 2;

template <int NT>
struct TgCfg {
    static constexpr int A_TERM = kTgM * kTgKC * 2;  // bytes of one BF16 term of the A chunk
    static constexpr int B_TERM = NT * kTgKC * 2;    // bytes of one BF16 term of the operator chunk
    static constexpr int STAGE = 3 * A_TERM + 3 * B_TERM;
    static constexpr size_t SMEM = (size_t)kTgStages * STAGE + 4 * 8 + 16;
    static constexpr int TMEM_COLS = tmem_alloc_cols(2 * NT);  // two chunk accumulators
};

struct TgParams {
    const float *src;
    float *dst;
    const long long *src_off, *dst_off;  // indexed arrays (element offsets), or null
    long long rows_total;                // arrays * R
    int R;                               // rows per array (1: the output is not transposed)
    int K, N;                            // contraction length (row length), output length
    int KC, nk;                          // K per chunk, chunks
    int n_tiles;                         // N / NT
    long long items;                     // row tiles * n_tiles
    const __nv_bfloat16 *ops;            // operator terms, [n tile][k chunk][term][NT x KC K-major]
    const float *lam;                    // optional: output (n, r) of an array times lam[n * R + r]
    unsigned int *status;
};

template <int NT, int TERMS>
__global__ void __launch_bounds__(128) k_tcg(const TgParams p)
{
    using C = TgCfg<NT>;
    extern __shared__ __align__(1024) uint8_t tgs[];
    uint64_t *bfull = reinterpret_cast<uint64_t *>(tgs + kTgStages * C::STAGE);  // operator chunk landed
    uint64_t *mdone = bfull + kTgStages;                                          // products of a stage done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + kTgStages);

    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < kTgStages; ++s) {
            mbar_init(&bfull[s], 1);
            mbar_init(&mdone[s], 1);
        }
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    pdl_launch_dependents();
    pdl_wait_prerequisites();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // chunk partials, double-buffered: accumulator a at TMEM column a * NT
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    const int KC = p.KC;
    const uint32_t sbo = (uint32_t)(KC / 8) * 128u;  // M/N-adjacent core matrices
    constexpr uint32_t idesc = tc_idesc(NT, false);
    const uint32_t b_term = (uint32_t)NT * KC * 2;  // bytes of one operator term of a chunk
    const uint32_t b_bytes = (uint32_t)TERMS * b_term;
    const long long b_chunk_elems = 3LL * NT * KC;

    // source row of this thread for a row tile (null beyond the last row)
    auto row_ptr = [&](long long item) -> const float * {
        const long long m = (item / p.n_tiles) * kTgM + tid;
        if (m >= p.rows_total) return nullptr;
        const long long b = m / p.R;
        const long long r = m - b * p.R;
        return p.src + (p.src_off ? p.src_off[b] : b * (long long)p.R * p.K) + r * p.K;
    };
    float v[kTgKC];
    auto load_chunk = [&](const float *row, int kc) {
        if (row) {
            const float4 *q = reinterpret_cast<const float4 *>(row + (long long)kc * KC);
#pragma unroll
            for (int i = 0; i < kTgKC / 4; ++i)
                if (4 * i < KC) {
                    const float4 t = __ldg(q + i);
                    v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
                }
        } else {
#pragma unroll
            for (int i = 0; i < kTgKC; ++i) v[i] = 0.0f;
        }
    };

    bool ok = true;
    uint32_t g = 0;                      // chunks this CTA has started
    long long last_b = -1, last_c = -1;  // thread 0: last operator copy and last commit issued
    float sum[NT];                       // this thread's row of the tile, summed over the chunks
#pragma unroll
    for (int j = 0; j < NT; ++j) sum[j] = 0.0f;
    // add the finished chunk partial in TMEM accumulator a to sum (in chunk order)
    auto take_partial = [&](int a) {
#pragma unroll
        for (int c = 0; c < NT / 16; ++c) {
            float y[16];
            tmem_ld16(tmem + (uint32_t)(a * NT) + lane_off + 16 * c, y);
#pragma unroll
            for (int j = 0; j < 16; ++j) sum[16 * c + j] += y[j];
        }
    };
    long long item = blockIdx.x;
    if (item < p.items) load_chunk(row_ptr(item), 0);
    for (; ok && item < p.items; item += gridDim.x) {
        const int nt = (int)(item % p.n_tiles);
        const float *row = row_ptr(item);
        for (int kc = 0; kc < p.nk; ++kc, ++g) {
            const int s = (int)(g & 1u);
            const uint32_t use = g >> 1;
            uint8_t *st = tgs + s * C::STAGE;
            // stage s and accumulator s are free once the products of chunk
            // g - 2 are done; that chunk's partial is added here when it belongs
            // to this item (the previous item's last two were added at its end)
            if (g >= 2) {
                if (!mbar_wait_bounded(&mdone[s], (use - 1) & 1u)) ok = false;
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
                if (ok && kc >= 2) {
                    tc_fence_after();
                    take_partial(s);
                }
            }
            if (tid == 0 && ok) {
                mbar_arrive_expect_tx(&bfull[s], b_bytes);
                bulk_load(st + 3 * C::A_TERM, p.ops + ((long long)nt * p.nk + kc) * b_chunk_elems, b_bytes, &bfull[s]);
                last_b = g;
            }
            if (ok) {
                // split this thread's row of the chunk into BF16 terms (K-major row tid)
#pragma unroll
                for (int q = 0; q < kTgKC / 8; ++q) {
                    if (8 * q < KC) {
                        __nv_bfloat16 t[TERMS][8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            __nv_bfloat16 sp[3];
                            split3<TERMS>(v[8 * q + e], sp);
#pragma unroll
                            for (int tt = 0; tt < TERMS; ++tt) t[tt][e] = sp[tt];
                        }
                        const int off = kmaj_off_bytes(tid, 8 * q, KC);
#pragma unroll
                        for (int tt = 0; tt < TERMS; ++tt)
                            *reinterpret_cast<uint4 *>(st + tt * C::A_TERM + off) = *reinterpret_cast<const uint4 *>(t[tt]);
                    }
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            ok = __syncthreads_and(ok);
            tc_fence_after();
            if (!ok) break;
            // prefetch the next chunk's row segment (the next item's first one
            // after the last chunk) while the products run
            {
                const long long ni = item + gridDim.x;
                if (kc + 1 < p.nk) load_chunk(row, kc + 1);
                else if (ni < p.items) load_chunk(row_ptr(ni), 0);
            }
            if (tid == 0) {
                if (!mbar_wait_bounded(&bfull[s], use & 1u)) {
                    record_timeout(p.status);  // the others learn of it at their next wait
                } else {
                    const uint32_t a0 = smem_u32(st), b0 = smem_u32(st + 3 * C::A_TERM);
                    // this chunk's products into a fresh accumulator: the small ones
                    // (term orders summing to 1 or 2) smallest first, the main one last
                    constexpr int pa[6] = {2, 1, 0, 1, 0, 0};
                    constexpr int pb[6] = {0, 1, 2, 0, 1, 0};
                    constexpr int first = TERMS == 3 ? 0 : (TERMS == 2 ? 3 : 5);
#pragma unroll
                    for (int pr = first; pr < 6; ++pr)
                        for (int ks = 0; ks < KC / 16; ++ks)
                            tc_mma(tmem + (uint32_t)(s * NT), smem_desc(a0 + pa[pr] * C::A_TERM + ks * 256, 128, sbo),
                                   smem_desc(b0 + pb[pr] * b_term + ks * 256, 128, sbo), idesc,
                                   (pr > first || ks > 0) ? 1u : 0u);
                    tc_commit(&mdone[s]);
                    last_c = g;
                }
            }
        }
        if (!ok) break;
        // ---- epilogue: the item's last two chunk partials, then this
        // thread's row of the tile (TMEM lane tid) is complete
        const uint32_t gl = g - 1;
        if (p.nk >= 2) {
            const uint32_t gp = g - 2;
            if (!mbar_wait_bounded(&mdone[gp & 1u], (gp >> 1) & 1u)) ok = false;
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                tc_fence_after();
                take_partial((int)(gp & 1u));
            }
        }
        if (ok && !mbar_wait_bounded(&mdone[gl & 1u], (gl >> 1) & 1u)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
            tc_fence_after();
            take_partial((int)(gl & 1u));
        }
        ok = __syncthreads_and(ok);
        if (!ok) break;
        const long long m = (item / p.n_tiles) * kTgM + tid;
        if (m < p.rows_total) {
            const long long b = m / p.R;
            const long long r = m - b * p.R;
            float *dbase = p.dst + (p.dst_off ? p.dst_off[b] : b * (long long)p.N * p.R);
            const int n0 = nt * NT;
            if (p.lam) {
#pragma unroll
                for (int j = 0; j < NT; ++j) sum[j] *= __ldg(p.lam + (long long)(n0 + j) * p.R + r);
            }
            if (p.R == 1) {
                float4 *d4 = reinterpret_cast<float4 *>(dbase + n0);
#pragma unroll
                for (int j = 0; j < NT / 4; ++j)
                    d4[j] = make_float4(sum[4 * j], sum[4 * j + 1], sum[4 * j + 2], sum[4 * j + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < NT; ++j) dbase[(long long)(n0 + j) * p.R + r] = sum[j];
            }
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) sum[j] = 0.0f;
        // every lane has read its accumulators before the next item's products overwrite them
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (!ok && tid == 0) {
        record_timeout(p.status);
        // error path: the last operator copy and the last committed products of
        // this CTA finish (each wait bounded) before its shared memory and TMEM
        // are released
        if (last_b >= 0) mbar_wait_bounded(&bfull[last_b & 1], (uint32_t)((last_b >> 1) & 1));
        if (last_c >= 0) mbar_wait_bounded(&mdone[last_c & 1], (uint32_t)((last_c >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
}

// ------------------------------------------------------------ warp-specialized kernel
// For long contractions the in-kernel split above re-splits every input row
// once per output tile and occupies the CUDA cores the whole time.  There the
// pass runs in two kernels: k_tg_presplit writes the three BF16 terms of the
// input once, already in the blocked canonical layout (block (row tile, K
// chunk) = three 128 x KC K-major terms), and k_tcg2 streams both operands
// with bulk copies:
//   warp 0, lane 0: producer -- one bulk copy of the input terms and one of
//     the operator terms per chunk into a two-stage ring (full / empty
//     mbarriers);
//   warp 1, lane 0: issues the six products of a chunk into one of four TMEM
//     partial accumulators and commits them twice (stage free, partial ready);
//   warps 2-5: each reads its TMEM lane quadrant (warp % 4) of a finished
//     partial, adds it to its row's running sums in registers (round to
//     nearest, chunk order), releases the partial, and at the end of a tile
//     stores the row transposed.
// Tiles are 128 rows by 128 outputs, K chunks of 64.

// Split src rows into the blocked BF16 terms: thread t of a group of eight
// takes row (8 q + t % 8) of a core matrix, so that eight lanes write one
// 128-byte core matrix and each lane reads one 32-byte sector.
template <int TERMS>
__global__ void k_tg_presplit(const float *src, const long long *src_off, long long rows_total, int R, int K, int KC,
                              long long m_tiles, __nv_bfloat16 *abuf)
{
    const int nk = K / KC;
    const int groups = KC / 8;                       // 8-column groups per chunk row
    const long long per_tile = 128LL * K / 8;        // work units per row tile
    const long long total = m_tiles * per_tile;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const long long mt = u / per_tile;
        long long rem = u - mt * per_tile;
        const int r8 = (int)(rem & 7);               // row within the core matrix
        rem >>= 3;
        const int kc = (int)(rem / (16LL * groups)); // chunk
        rem -= (long long)kc * 16 * groups;
        const int g = (int)(rem % groups);           // 8-column group within the chunk
        const int rq = (int)(rem / groups);          // core-matrix row block (0..15)
        const int row = rq * 8 + r8;                 // row within the tile
        const long long m = mt * 128 + row;
        float v[8];
        if (m < rows_total) {
            const long long b = m / R, r = m - b * R;
            const float *q = src + (src_off ? src_off[b] : b * (long long)R * K) + r * K + (long long)kc * KC + 8 * g;
            const float4 t0 = __ldg(reinterpret_cast<const float4 *>(q));
            const float4 t1 = __ldg(reinterpret_cast<const float4 *>(q) + 1);
            v[0] = t0.x; v[1] = t0.y; v[2] = t0.z; v[3] = t0.w;
            v[4] = t1.x; v[5] = t1.y; v[6] = t1.z; v[7] = t1.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = 0.0f;
        }
        __nv_bfloat16 t[TERMS][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            __nv_bfloat16 sp[3];
            split3<TERMS>(v[e], sp);
#pragma unroll
            for (int tt = 0; tt < TERMS; ++tt) t[tt][e] = sp[tt];
        }
        uint8_t *blk = reinterpret_cast<uint8_t *>(abuf) + (mt * nk + kc) * (3LL * 128 * KC * 2);
        const int off = kmaj_off_bytes(row, 8 * g, KC);
#pragma unroll
        for (int tt = 0; tt < TERMS; ++tt)
            *reinterpret_cast<uint4 *>(blk + (long long)tt * 128 * KC * 2 + off) = *reinterpret_cast<const uint4 *>(t[tt]);
    }
}

constexpr int kTg2NT = 128;
constexpr int kTg2Stages = 2;
// TMEM partial accumulators (kTg2Acc x 128 columns of the 512): the MMA lane
// may run kTg2Acc - 1 chunks ahead of the epilogue warps' reads
constexpr int kTg2Acc = 4;
static_assert(tmem_alloc_cols(kTg2Acc * 128) == kTg2Acc * 128 && kTg2Acc * 128 <= 512, "TMEM allocation");
constexpr int kTg2AStage = 3 * 128 * kTgKC * 2;       // bytes of the input terms of a chunk
constexpr int kTg2BStage = 3 * kTg2NT * kTgKC * 2;    // bytes of the operator terms of a chunk
constexpr int kTg2Stage = kTg2AStage + kTg2BStage;
constexpr size_t kTg2Smem = (size_t)kTg2Stages * kTg2Stage + (2 * kTg2Stages + 2 * kTg2Acc) * 8 + 16;

struct Tg2Params {
    const __nv_bfloat16 *abuf;       // input terms, [row tile][chunk][term][128 x KC]
    const __nv_bfloat16 *ops;        // operator terms, [n tile][chunk][term][128 x KC]
    float *dst;
    const long long *dst_off;
    long long rows_total;
    int R, N, KC, nk, n_tiles;
    long long items;
    const float *lam;
    unsigned int *status;
};

template <int TERMS>
__global__ void __launch_bounds__(192, 1) k_tcg2(const Tg2Params p)
{
    extern __shared__ __align__(1024) uint8_t t2s[];
    uint64_t *full = reinterpret_cast<uint64_t *>(t2s + kTg2Stages * kTg2Stage);
    uint64_t *empty = full + kTg2Stages;
    uint64_t *pfull = empty + kTg2Stages;   // partial accumulator ready
    uint64_t *pempty = pfull + kTg2Acc;     // partial accumulator read
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(pempty + kTg2Acc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kTg2Stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < kTg2Acc; ++a) {
            mbar_init(&pfull[a], 1);
            mbar_init(&pempty[a], 4);  // one arrival per epilogue warp
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTg2Acc * kTg2NT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    pdl_launch_dependents();
    pdl_wait_prerequisites();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int KC = p.KC, nk = p.nk;
    const uint32_t a_term = 128u * KC * 2, b_term = (uint32_t)kTg2NT * KC * 2;
    const long long blk_elems = 3LL * 128 * KC;  // input and operator blocks alike (NT = 128)
    long long last_load = -1, last_commit = -1;  // error path: the last copy and commit issued
    bool ok = true;

    if (warp == 0) {
        // ---- producer
        if (lane == 0) {
            long long c = 0;
            for (long long item = blockIdx.x; ok && item < p.items; item += gridDim.x) {
                const long long mt = item / p.n_tiles;
                const int nt = (int)(item % p.n_tiles);
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int s = (int)(c % kTg2Stages);
                    const uint32_t use = (uint32_t)(c / kTg2Stages);
                    if (c >= kTg2Stages && !mbar_wait_bounded(&empty[s], (use - 1) & 1u)) { ok = false; break; }
                    if (*abort_flag) { ok = false; break; }
                    uint8_t *st = t2s + s * kTg2Stage;
                    mbar_arrive_expect_tx(&full[s], (uint32_t)TERMS * (a_term + b_term));
                    bulk_load(st, p.abuf + (mt * nk + kc) * blk_elems, (uint32_t)TERMS * a_term, &full[s]);
                    bulk_load(st + kTg2AStage, p.ops + ((long long)nt * nk + kc) * blk_elems, (uint32_t)TERMS * b_term,
                              &full[s]);
                    last_load = c;
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue
        if (lane == 0) {
            constexpr uint32_t idesc = tc_idesc(kTg2NT, false);
            const uint32_t sbo = (uint32_t)(KC / 8) * 128u;
            constexpr int pa[6] = {2, 1, 0, 1, 0, 0};
            constexpr int pb[6] = {0, 1, 2, 0, 1, 0};
            constexpr int first = TERMS == 3 ? 0 : (TERMS == 2 ? 3 : 5);
            long long c = 0;
            for (long long item = blockIdx.x; ok && item < p.items; item += gridDim.x) {
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int s = (int)(c % kTg2Stages), a = (int)(c % kTg2Acc);
                    if (!mbar_wait_bounded(&full[s], (uint32_t)(c / kTg2Stages) & 1u)) { ok = false; break; }
                    if (c >= kTg2Acc && !mbar_wait_bounded(&pempty[a], (uint32_t)(c / kTg2Acc - 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    if (*abort_flag) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(t2s + s * kTg2Stage), b0 = a0 + kTg2AStage;
                    const uint32_t d = tmem + (uint32_t)(a * kTg2NT);
#pragma unroll
                    for (int pr = first; pr < 6; ++pr)
                        for (int ks = 0; ks < KC / 16; ++ks)
                            tc_mma(d, smem_desc(a0 + pa[pr] * a_term + ks * 256, 128, sbo),
                                   smem_desc(b0 + pb[pr] * b_term + ks * 256, 128, sbo), idesc,
                                   (pr > first || ks > 0) ? 1u : 0u);
                    tc_commit(&empty[s]);
                    tc_commit(&pfull[a]);
                    last_commit = c;
                }
            }
        }
    } else {
        // ---- epilogue: TMEM lane quadrant q of every partial
        const int q = warp & 3;
        const int row = 32 * q + lane;
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        float sum[kTg2NT];
#pragma unroll
        for (int j = 0; j < kTg2NT; ++j) sum[j] = 0.0f;
        long long c = 0;
        for (long long item = blockIdx.x; ok && item < p.items; item += gridDim.x) {
            for (int kc = 0; kc < nk; ++kc, ++c) {
                const int a = (int)(c % kTg2Acc);
                bool w = mbar_wait_bounded(&pfull[a], (uint32_t)(c / kTg2Acc) & 1u);
                w = __all_sync(0xffffffffu, w);
                if (!w) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int cc = 0; cc < kTg2NT / 16; ++cc) {
                    float y[16];
                    tmem_ld16(tmem + (uint32_t)(a * kTg2NT) + lane_off + 16 * cc, y);
#pragma unroll
                    for (int j = 0; j < 16; ++j) sum[16 * cc + j] += y[j];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&pempty[a]);
            }
            if (!ok) break;
            const long long m = (item / p.n_tiles) * 128 + row;
            if (m < p.rows_total) {
                const long long b = m / p.R, r = m - b * p.R;
                float *dbase = p.dst + (p.dst_off ? p.dst_off[b] : b * (long long)p.N * p.R);
                const int n0 = (int)(item % p.n_tiles) * kTg2NT;
                if (p.lam) {
#pragma unroll
                    for (int j = 0; j < kTg2NT; ++j) sum[j] *= __ldg(p.lam + (long long)(n0 + j) * p.R + r);
                }
#pragma unroll
                for (int j = 0; j < kTg2NT; ++j) dbase[(long long)(n0 + j) * p.R + r] = sum[j];
            }
#pragma unroll
            for (int j = 0; j < kTg2NT; ++j) sum[j] = 0.0f;
        }
    }
    if (!ok) {
        *abort_flag = 1;
        if (lane == 0) record_timeout(p.status);
    }
    // error path: the issuing lanes wait (bounded) for their last copy and
    // their last products before the CTA releases shared memory and TMEM
    if (warp == 0 && lane == 0 && last_load >= 0)
        mbar_wait_bounded(&full[last_load % kTg2Stages], (uint32_t)(last_load / kTg2Stages) & 1u);
    if (warp == 1 && lane == 0 && last_commit >= 0)
        mbar_wait_bounded(&pfull[last_commit % kTg2Acc], (uint32_t)(last_commit / kTg2Acc) & 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTg2Acc * kTg2NT)
                     : "memory");
}

// ------------------------------------------------------------ 8 x 8 arrays
// One product per direction with the 64 x 64 Kronecker operator over the
// vectorized array (row-major 8 x 8 = 64 values), warp-specialized like
// k_tcg2: tiles of 128 arrays (the MMA's M), K = N = 64.
//   warps 0-3: each thread owns one array of the tile: cp.async copies of its
//     64 values two tiles ahead into a padded row slot, the BF16 split into
//     the K-major operand (row = array);
//   warp 4, lane 0: the six products of a tile into one of two TMEM
//     accumulators;
//   warps 5-8: read the array's 64 outputs from TMEM (lane quadrant warp % 4),
//     optionally times the diagonal, and store them (256 contiguous bytes).
struct KronParams {
    const float *src;
    float *dst;
    const long long *src_off, *dst_off;
    long long count;                 // arrays
    int ntiles;
    const __nv_bfloat16 *ops;        // three terms of the 64 x 64 operator, K-major
    const float *lam;                // optional: output n of an array times lam[n]
    unsigned int *status;
};

constexpr int kKronNS = 2;                        // operand stages and accumulators
constexpr int kKronD = 2;                         // input tiles in flight per loading thread
constexpr int kKronATerm = 128 * 64 * 2;          // bytes of one BF16 term of a tile
constexpr int kKronBBytes = 3 * 64 * 64 * 2;
constexpr int kKronXP = 68;                       // padded row slot (floats)
constexpr int kKronXBytes = kKronD * 128 * kKronXP * 4;
constexpr int kKronNBar = 4 * kKronNS + 1;
constexpr size_t kKronSmem = (size_t)kKronNS * 3 * kKronATerm + kKronBBytes + kKronXBytes + kKronNBar * 8 + 16;
constexpr int kKronTmem = tmem_alloc_cols(kKronNS * 64);

template <int TERMS>
__global__ void __launch_bounds__(288, 1) k_tc_kron(const KronParams p)
{
    extern __shared__ __align__(1024) uint8_t ksm[];
    uint8_t *abuf = ksm;
    uint8_t *bop = ksm + kKronNS * 3 * kKronATerm;
    float *xring = reinterpret_cast<float *>(bop + kKronBBytes);
    uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(xring) + kKronXBytes);
    uint64_t *a_full = bar, *a_empty = bar + kKronNS, *d_full = bar + 2 * kKronNS, *d_empty = bar + 3 * kKronNS;
    uint64_t *b_full = bar + 4 * kKronNS;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + kKronNBar);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < kKronNS; ++i) {
            mbar_init(&a_full[i], 128);
            mbar_init(&a_empty[i], 1);
            mbar_init(&d_full[i], 1);
            mbar_init(&d_empty[i], 128);
        }
        mbar_init(b_full, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kKronTmem)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    pdl_launch_dependents();
    pdl_wait_prerequisites();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int ntl = p.ntiles > (int)blockIdx.x ? (p.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                                               : 0;
    bool ok = true;
    long long last_commit = -1;

    if (warp < 4) {
        // ---- loading and splitting: thread tid owns array (tile * 128 + tid)
        auto arr_of = [&](int t) -> long long { return ((long long)blockIdx.x + (long long)t * gridDim.x) * 128 + tid; };
        auto issue = [&](int t) {
            if (t < ntl) {
                const long long a = arr_of(t);
                if (a < p.count) {
                    const float *src = p.src + (p.src_off ? p.src_off[a] : a * 64);
                    float *dst = xring + ((t % kKronD) * 128 + tid) * kKronXP;
#pragma unroll
                    for (int q = 0; q < 16; ++q) cp_async16(dst + 4 * q, src + 4 * q);
                }
            }
            cp_async_commit();  // one group per tile, empty past the end
        };
#pragma unroll 1
        for (int t = 0; t < kKronD; ++t) issue(t);
        float v[64];
        for (int t = 0; t < ntl; ++t) {
            cp_async_wait_group<kKronD - 1>();
            if (arr_of(t) < p.count) {
                const float4 *q4 = reinterpret_cast<const float4 *>(xring + ((t % kKronD) * 128 + tid) * kKronXP);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float4 x = q4[q];
                    v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 64; ++j) v[j] = 0.0f;
            }
            issue(t + kKronD);
            const int s = t % kKronNS;
            if (t >= kKronNS && !mbar_wait_bounded(&a_empty[s], (uint32_t)(t / kKronNS - 1) & 1u)) { ok = false; break; }
            if (*abort_flag) { ok = false; break; }
            uint8_t *st = abuf + s * 3 * kKronATerm;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                __nv_bfloat16 tt[TERMS][8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    __nv_bfloat16 sp[3];
                    split3<TERMS>(v[8 * q + e], sp);
#pragma unroll
                    for (int k = 0; k < TERMS; ++k) tt[k][e] = sp[k];
                }
                const int off = kmaj_off_bytes(tid, 8 * q, 64);
#pragma unroll
                for (int k = 0; k < TERMS; ++k)
                    *reinterpret_cast<uint4 *>(st + k * kKronATerm + off) = *reinterpret_cast<const uint4 *>(tt[k]);
            }
            fence_proxy_async_smem();
            mbar_arrive(&a_full[s]);
        }
        cp_async_wait_all();
    } else if (warp == 4) {
        // ---- MMA issue
        if (lane == 0) {
            mbar_arrive_expect_tx(b_full, kKronBBytes);
            bulk_load(bop, p.ops, kKronBBytes, b_full);
            if (!mbar_wait_bounded(b_full, 0)) ok = false;
            constexpr uint32_t idesc = tc_idesc(64, false);
            constexpr uint32_t sbo = 8 * 128;  // K = 64: eight core matrices along K
            constexpr int pa[6] = {2, 1, 0, 1, 0, 0};
            constexpr int pb[6] = {0, 1, 2, 0, 1, 0};
            constexpr int first = TERMS == 3 ? 0 : (TERMS == 2 ? 3 : 5);
            const uint32_t b0 = smem_u32(bop);
            for (int t = 0; ok && t < ntl; ++t) {
                const int s = t % kKronNS;
                if (!mbar_wait_bounded(&a_full[s], (uint32_t)(t / kKronNS) & 1u) ||
                    (t >= kKronNS && !mbar_wait_bounded(&d_empty[s], (uint32_t)(t / kKronNS - 1) & 1u)) || *abort_flag) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(abuf + s * 3 * kKronATerm);
                const uint32_t d = tmem + (uint32_t)(s * 64);
#pragma unroll
                for (int pr = first; pr < 6; ++pr)
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        tc_mma(d, smem_desc(a0 + pa[pr] * kKronATerm + ks * 256, 128, sbo),
                               smem_desc(b0 + pb[pr] * (64 * 64 * 2) + ks * 256, 128, sbo), idesc,
                               (pr > first || ks > 0) ? 1u : 0u);
                tc_commit(&a_empty[s]);
                tc_commit(&d_full[s]);
                last_commit = t;
            }
        }
    } else {
        // ---- TMEM read and store: thread = array (32 * (warp % 4) + lane) of the tile
        const int row = 32 * (warp & 3) + lane;
        const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
        float y[64];
        for (int t = 0; t < ntl; ++t) {
            const int s = t % kKronNS;
            bool w = mbar_wait_bounded(&d_full[s], (uint32_t)(t / kKronNS) & 1u) && !*abort_flag;
            w = __all_sync(0xffffffffu, w);
            if (!w) { ok = false; break; }
            tc_fence_after();
#pragma unroll
            for (int c = 0; c < 4; ++c) tmem_ld16(tmem + (uint32_t)(s * 64) + lane_off + 16 * c, y + 16 * c);
            tc_fence_before();
            mbar_arrive(&d_empty[s]);
            const long long a = ((long long)blockIdx.x + (long long)t * gridDim.x) * 128 + row;
            if (a < p.count) {
                if (p.lam) {
#pragma unroll
                    for (int j = 0; j < 64; ++j) y[j] *= __ldg(p.lam + j);
                }
                float4 *d4 = reinterpret_cast<float4 *>(p.dst + (p.dst_off ? p.dst_off[a] : a * 64));
#pragma unroll
                for (int q = 0; q < 16; ++q) d4[q] = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
            }
        }
    }
    if (!ok) {
        *abort_flag = 1;
        if (lane == 0) record_timeout(p.status);
    }
    // error path: the MMA lane waits (bounded) for the operator copy and its
    // last committed products before shared memory and TMEM are released
    if (warp == 4 && lane == 0 && !ok) {
        mbar_wait_bounded(b_full, 0);
        if (last_commit >= 0)
            mbar_wait_bounded(&d_full[last_commit % kKronNS], (uint32_t)(last_commit / kKronNS) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kKronTmem) : "memory");
}

template <int TERMS>
static cudaError_t kron_launch(const KronParams &p0, cudaStream_t stream)
{
    static DeviceLaunchCache cache;
    int dev = 0, bps = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    auto kern = k_tc_kron<TERMS>;
    e = cache.get(
        dev,
        [&](int d, int &b, int &n) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKronSmem);
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
            b = 1;
            if (r == cudaSuccess && debug_enabled())
                fprintf(stderr, "[bdct] k_tc_kron<%d>: 1 CTA/SM x 288 threads, smem %zu B, TMEM %d cols\n", TERMS,
                        kKronSmem, kKronTmem);
            return r;
        },
        &bps, &sms);
    if (e != cudaSuccess) return e;
    KronParams p = p0;
    long long grid = sms;
    if (grid > p.ntiles) grid = p.ntiles;
    if (grid <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(288);
    cfg.dynamicSmemBytes = kKronSmem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

// ------------------------------------------------------------ operator tables
// Operator M (N = K = n, or the 64 x 64 Kronecker operator of 8 x 8 arrays)
// for direction 1 (forward: M[f][j] = s_f cos(pi (2j+1) f / 2n)) or 2
// (inverse: M[j][f] = s_f cos(...)), s the scale of Eq. 1 (orthonormal) or of
// the REDFT pair; split in FP64 into three BF16 terms and written blocked for
// the kernel: block (n tile, k chunk) holds the three terms of its NT x KC
// piece, each in the canonical K-major layout.
__device__ double tg_op_value(int row, int col, int n, int direction, int norm)
{
    const int f = direction == 1 ? row : col;  // frequency index
    const int j = direction == 1 ? col : row;  // sample index
    double s;
    if (norm == 0) s = (f == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
    else if (direction == 1) s = 2.0;
    else s = (f == 0) ? 1.0 : 2.0;
    // cos(pi m / (2n)) with the argument reduced exactly
    const long long m = (2LL * j + 1) * f;
    const long long d = 2LL * n;
    long long red = m % (2 * d);
    if (red > d) red = 2 * d - red;
    double sign = 1.0;
    if (2 * red > d) { red = d - red; sign = -1.0; }
    double c;
    if (red == 0) c = sign;
    else if (2 * red == d) c = 0.0;
    else c = sign * cospi((double)red / (double)d);
    return s * c;
}

__global__ void k_gen_tg_op(__nv_bfloat16 *dst, int N, int K, int direction, int norm, int NT, int KC, int kron)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * K) return;
    const int nn = (int)(idx / K), kk = (int)(idx % K);
    double val;
    if (kron) {
        // (Q (x) Q)[(f1, f2)][(i, j)] = M8[f1][i] * M8[f2][j] for the row-major 8 x 8 array
        val = tg_op_value(nn >> 3, kk >> 3, 8, direction, norm) * tg_op_value(nn & 7, kk & 7, 8, direction, norm);
    } else {
        val = tg_op_value(nn, kk, N, direction, norm);
    }
    const __nv_bfloat16 t0 = __double2bfloat16(val);
    const double r1 = val - (double)__bfloat162float(t0);
    const __nv_bfloat16 t1 = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(t1);
    const __nv_bfloat16 t2 = __double2bfloat16(r2);
    const long long blk = (long long)(nn / NT) * (K / KC) + kk / KC;
    const long long base = blk * 3LL * NT * KC + kmaj_off_bytes(nn % NT, kk % KC, KC) / 2;
    dst[base] = t0;
    dst[base + (long long)NT * KC] = t1;
    dst[base + 2LL * NT * KC] = t2;
}

// Contractions of at least this length run on the warp-specialized kernel
// (input split beforehand, 128-wide tiles); shorter ones split in the kernel.
constexpr int kTg2MinK = 128;

static bool tg_use_v2(int n) { return n >= kTg2MinK && n % 128 == 0; }

// Tile width for an output length: 128 on the warp-specialized kernel, else
// the largest of 64, 32, 16 dividing it (a thread of the single-role kernel
// holds its row of the tile in registers across the K loop).
static int tg_nt(int n)
{
    if (tg_use_v2(n)) return 128;
    for (int nt : {64, 32, 16})
        if (n % nt == 0) return nt;
    return 0;
}

// K chunk for a contraction length: 64 for multiples of 64, else the length
// itself (16 or 32).
static int tg_kc(int k) { return k % 64 == 0 ? 64 : ((k == 16 || k == 32) ? k : 0); }

bool tg_axis_ok(int n) { return n == 16 || n == 32 || (n % 64 == 0 && n >= 64 && n <= 8192); }

size_t tg_table_elems(int n) { return (size_t)3 * n * n; }

cudaError_t tg_gen_table(__nv_bfloat16 *dst, int n, int direction, int norm, bool kron, cudaStream_t s)
{
    const int N = kron ? 64 : n;
    const int NT = tg_nt(N), KC = tg_kc(N);
    if (!NT || !KC) return cudaErrorInvalidValue;
    const long long total = (long long)N * N;
    k_gen_tg_op<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(dst, N, N, direction, norm, NT, KC, kron ? 1 : 0);
    return cudaGetLastError();
}

template <int NT, int TERMS>
static cudaError_t tg_launch_one(const TgParams &p0, cudaStream_t stream)
{
    using C = TgCfg<NT>;
    auto kern = k_tcg<NT, TERMS>;
    static DeviceLaunchCache cache;
    int dev = 0, blocks_per_sm = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cache.get(
        dev,
        [&](int d, int &bps, int &sms) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
            if (r != cudaSuccess) return r;
            // resident CTAs from shared memory, capped by TMEM (512 columns per
            // SM) and threads; the runtime's occupancy query does not see TMEM
            int smem_per_sm = 0, reserved = 0;
            cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, d);
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, d);
            int occ = (int)((size_t)smem_per_sm / (C::SMEM + (size_t)reserved));
            const int tmem_cap = 512 / C::TMEM_COLS;
            if (occ > tmem_cap) occ = tmem_cap;
            if (occ > 16) occ = 16;
            bps = occ;
            r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
            if (r != cudaSuccess) return r;
            if (bps < 1) return cudaErrorInvalidConfiguration;
            if (debug_enabled())
                fprintf(stderr, "[bdct] k_tcg<%d,%d>: %d CTAs/SM, smem %zu B, TMEM %d cols\n", NT, TERMS, bps,
                        C::SMEM, C::TMEM_COLS);
            return cudaSuccess;
        },
        &blocks_per_sm, &num_sms);
    if (e != cudaSuccess) return e;
    TgParams p = p0;
    long long grid = (long long)blocks_per_sm * num_sms;
    if (grid > p.items) grid = p.items;
    if (grid <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int NT>
static cudaError_t tg_launch_nt(int terms, const TgParams &p, cudaStream_t s)
{
    switch (terms) {
        case 3: return tg_launch_one<NT, 3>(p, s);
        case 2: return tg_launch_one<NT, 2>(p, s);
        default: return tg_launch_one<NT, 1>(p, s);
    }
}

size_t tg_split_elems(long long rows, int K)
{
    const long long m_tiles = (rows + 127) / 128;
    return (size_t)m_tiles * 128 * (size_t)K * 3;
}

template <int TERMS>
static cudaError_t tg2_launch(const float *src, const long long *src_off, const Tg2Params &p0, int K,
                              __nv_bfloat16 *abuf, cudaStream_t stream)
{
    static DeviceLaunchCache cache;
    int dev = 0, bps = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    auto kern = k_tcg2<TERMS>;
    e = cache.get(
        dev,
        [&](int d, int &b, int &n) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTg2Smem);
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
            b = 1;
            if (r == cudaSuccess && debug_enabled())
                fprintf(stderr, "[bdct] k_tcg2<%d>: 1 CTA/SM x 192 threads, smem %zu B, TMEM %d cols\n", TERMS,
                        kTg2Smem, kTg2Acc * kTg2NT);
            return r;
        },
        &bps, &sms);
    if (e != cudaSuccess) return e;
    Tg2Params p = p0;
    const long long m_tiles = (p.rows_total + 127) / 128;
    // 1. the input's BF16 terms, once
    {
        const long long work = m_tiles * 128LL * K / 8;
        long long blocks = (work + 255) / 256;
        if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
        k_tg_presplit<TERMS><<<(unsigned)blocks, 256, 0, stream>>>(src, src_off, p.rows_total, p.R, K, p.KC, m_tiles,
                                                                    abuf);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // 2. the products, persistent CTAs over the tiles
    p.abuf = abuf;
    long long grid = (long long)sms;
    if (grid > p.items) grid = p.items;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(192);
    cfg.dynamicSmemBytes = kTg2Smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

cudaError_t tg_pass(const float *src, float *dst, const long long *src_off, const long long *dst_off, long long count,
                    int R, int K, const __nv_bfloat16 *ops, int terms, const float *lam, __nv_bfloat16 *abuf,
                    unsigned int *status, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    const int N = K;  // square 1D operators (the Kronecker one included)
    const int NT = tg_nt(N), KC = tg_kc(K);
    if (!NT || !KC || R < 1) return cudaErrorInvalidValue;
    if (src == dst) return cudaErrorInvalidValue;  // a pass never runs in place
    if (R == 1 && K == 64) {
        // 8 x 8 arrays: the Kronecker pass (the table of a 64-point operator
        // is one block: the three terms in the K-major layout)
        const long long nt = (count + 127) / 128;
        if (nt > 0x7ff00000LL) return cudaErrorInvalidValue;
        KronParams kp{src, dst, src_off, dst_off, count, (int)nt, ops, lam, status};
        switch (terms) {
            case 3: return kron_launch<3>(kp, stream);
            case 2: return kron_launch<2>(kp, stream);
            default: return kron_launch<1>(kp, stream);
        }
    }
    if (tg_use_v2(K)) {
        if (!abuf) return cudaErrorInvalidValue;
        Tg2Params p{};
        p.ops = ops;
        p.dst = dst;
        p.dst_off = dst_off;
        p.rows_total = count * R;
        p.R = R;
        p.N = N;
        p.KC = KC;
        p.nk = K / KC;
        p.n_tiles = N / kTg2NT;
        p.items = ((p.rows_total + 127) / 128) * p.n_tiles;
        p.lam = lam;
        p.status = status;
        switch (terms) {
            case 3: return tg2_launch<3>(src, src_off, p, K, abuf, stream);
            case 2: return tg2_launch<2>(src, src_off, p, K, abuf, stream);
            default: return tg2_launch<1>(src, src_off, p, K, abuf, stream);
        }
    }
    TgParams p{};
    p.src = src;
    p.dst = dst;
    p.src_off = src_off;
    p.dst_off = dst_off;
    p.rows_total = count * R;
    p.R = R;
    p.K = K;
    p.N = N;
    p.KC = KC;
    p.nk = K / KC;
    p.n_tiles = N / NT;
    p.items = ((p.rows_total + kTgM - 1) / kTgM) * p.n_tiles;
    p.ops = ops;
    p.lam = lam;
    p.status = status;
    switch (NT) {
        case 64: return tg_launch_nt<64>(terms, p, stream);
        case 32: return tg_launch_nt<32>(terms, p, stream);
        default: return tg_launch_nt<16>(terms, p, stream);
    }
}

}  // namespace bdct
