// Split-BF16 tensor-core 2D DCT: C X C^T on tcgen05 with FP32 accumulation.
//
// What is computed: Eq. 2 of the BRiDCT paper as two dense contractions,
// Y = M_h X M_w^T, with M the 1D operator of the direction (Q_n of Eq. 1 for
// the orthonormal forward transform, Q_n^T for the inverse, the REDFT pair for
// the unnormalized setting); the round trip chains the forward and the
// inverse (four contractions).  Direct matrix evaluation costs n
// multiply-adds per point (Section 1.2); here the tensor cores take them.
//
// Exactness with BF16 operands (the paper excludes approximated matrices,
// Section 1.1): every FP32 operand x is split into BF16 terms
// x = x0 + x1 + x2 (each the round-to-nearest BF16 of the remaining residual,
// together holding the 24-bit significand), the FP64 operator matrix likewise,
// and the products x_a * m_b with a + b <= 2 are accumulated in FP32, smallest
// first.  Three terms and six products reach FP32 accuracy; the report-only
// variants keep two terms and three products (hi/lo) or one term and one
// product.
//
// Organization for an n x n array (n = 16, 32, 64), 128 threads per CTA:
// a tile stacks 128/n arrays so that thread t owns stack row t and TMEM lane
// t.  Pass 1: A = the rows of X (K-major, K = column index), B = M_w
// (K-major), D1[row][l] = T row in TMEM.  Pass 2 contracts over the row index:
// each thread re-splits its T row and stores it as the MN-major A operand
// (stack rows become the M dimension), B = M_h, D2[(array, l)][k] = Y[k][l];
// thread (array, l) then holds column l of Y and stores it coalesced across
// lanes.  Odd passes use K-major A, even passes MN-major A, which is what lets
// every pass start from values a thread already holds.
//
// Shared-memory operand layout (no swizzle), verified on the device: core
// matrices of 8 rows x 16 bytes stored as 128 contiguous bytes; the
// descriptor's leading byte offset is the stride between core matrices along
// K and the stride byte offset the stride along M/N, for both operand majors.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bdct_internal.h"
#include "ptx.cuh"
#include "tc_ptx.cuh"

#include <cstdio>

namespace bdct {

// ------------------------------------------------------------ kernel
template <int N>
struct TcCfg {
    static constexpr int G = 128 / N;               // arrays per tile
    static constexpr int A_TERM_BYTES = 128 * N * 2;
    static constexpr int B_TERM_BYTES = N * N * 2;
    static constexpr int KSTEPS = N / 16;
    static constexpr int KMAJ_SBO = (N / 8) * 128;  // M/N-adjacent core stride, K-major
    static constexpr int MN_LBO = 16 * 128;         // K-adjacent core stride, MN-major (M = 128)
    static constexpr int TMEM_COLS = tmem_alloc_cols(2 * N);
};

struct TcParams {
    const float *in;
    float *out;
    long long count;          // arrays (contiguous) or tiles (tiled)
    int tiles_per_row;        // tiled only
    int chunks_per_row;       // tiled only: ceil(tiles_per_row / G)
    long long ld_in, ld_out;  // tiled only
    int ntiles;
    const __nv_bfloat16 *ops;  // operator term tables, [op][term][B layout]
    const float *lam;          // spectral only: the N x N diagonal Lambda[k][l]
    unsigned int *status;
    const long long *in_off, *out_off;  // indexed batch, or null
};

// Byte offset of element (m, k) of an MN-major operand with M = 128 rows.
__device__ __forceinline__ int mnmaj_off_bytes(int m, int k)
{
    return (((k >> 3) * 16 + (m >> 3)) << 7) + ((k & 7) << 4) + ((m & 7) << 1);
}

// Write this thread's N values as split terms into the A buffer: K-major row
// `row` (values along K), or MN-major column `col` of rows base .. base+N-1.
template <int N, int TERMS, bool MN>
__device__ __forceinline__ void stage_a(uint8_t *a_buf, const float *v, int row_or_col, int base)
{
    using C = TcCfg<N>;
#pragma unroll
    for (int q = 0; q < N / 8; ++q) {
        __nv_bfloat16 t[TERMS][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            __nv_bfloat16 s[3];
            split3<TERMS>(v[8 * q + e], s);
#pragma unroll
            for (int tt = 0; tt < TERMS; ++tt) t[tt][e] = s[tt];
        }
        int off;
        if constexpr (!MN) off = kmaj_off_bytes(row_or_col, 8 * q, N);
        else off = mnmaj_off_bytes(base + 8 * q, row_or_col);
#pragma unroll
        for (int tt = 0; tt < TERMS; ++tt)
            *reinterpret_cast<uint4 *>(a_buf + tt * C::A_TERM_BYTES + off) = *reinterpret_cast<const uint4 *>(t[tt]);
    }
}

// Issue one pass: D = sum over products of A_ta * B_tb^T, smallest first.
template <int N, int TERMS, bool MN>
__device__ __forceinline__ void issue_pass(uint32_t a_base, uint32_t b_base, uint32_t d_tmem)
{
    using C = TcCfg<N>;
    constexpr uint32_t idesc = tc_idesc(N, MN);
    constexpr int NP = TERMS == 3 ? 6 : (TERMS == 2 ? 3 : 1);
    // products (a, b) with a + b <= TERMS - 1, smallest terms first
    constexpr int pa[6] = {2, 1, 0, 1, 0, 0};
    constexpr int pb[6] = {0, 1, 2, 0, 1, 0};
    constexpr int first = 6 - NP;
    bool acc = false;
#pragma unroll
    for (int p = first; p < 6; ++p) {
#pragma unroll
        for (int ks = 0; ks < C::KSTEPS; ++ks) {
            uint64_t da;
            if constexpr (!MN) da = smem_desc(a_base + pa[p] * C::A_TERM_BYTES + ks * 256, 128, C::KMAJ_SBO);
            else da = smem_desc(a_base + pa[p] * C::A_TERM_BYTES + ks * 2 * C::MN_LBO, C::MN_LBO, 128);
            const uint64_t db = smem_desc(b_base + pb[p] * C::B_TERM_BYTES + ks * 256, 128, C::KMAJ_SBO);
            tc_mma(d_tmem, da, db, idesc, acc ? 1u : 0u);
            acc = true;
        }
    }
}

template <int N, bool TILED>
__device__ __forceinline__ void tile_geom(const TcParams &p, int tile, long long &first, int &n, long long &brow,
                                          int &t0)
{
    using C = TcCfg<N>;
    if constexpr (!TILED) {
        first = (long long)tile * C::G;
        const long long rem = p.count - first;
        n = rem < C::G ? (int)rem : C::G;
        brow = 0;
        t0 = 0;
    } else {
        const unsigned int br = (unsigned int)tile / (unsigned int)p.chunks_per_row;
        brow = br;
        t0 = (int)((unsigned int)tile - br * (unsigned int)p.chunks_per_row) * C::G;
        const int rem = p.tiles_per_row - t0;
        n = rem < C::G ? rem : C::G;
        first = 0;
    }
}

// NPASS = 2 (forward or inverse; ops 0, 0) or 4 (round trip; ops 0, 0, 1, 1).
// SPEC (with NPASS = 4): the spectral composition of Prop. 1 -- after the
// second product every coefficient is multiplied by Lambda (the operators are
// the orthonormal forward and inverse, so the plain diagonal applies).
template <int N, int NPASS, int TERMS, bool TILED, bool SPEC = false>
__global__ void __launch_bounds__(128) k_tc_split(const TcParams p)
{
    using C = TcCfg<N>;
    constexpr int NOPS = NPASS / 2;
    extern __shared__ __align__(1024) uint8_t tsm[];
    uint8_t *a_buf = tsm;                                   // TERMS A terms
    uint8_t *b_buf = tsm + TERMS * C::A_TERM_BYTES;         // NOPS x 3 B terms
    uint64_t *bar = reinterpret_cast<uint64_t *>(b_buf + NOPS * 3 * C::B_TERM_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2);

    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bar[0], 1);  // MMA completion
        mbar_init(&bar[1], 1);  // operator tables landed
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
    const uint32_t d_tmem[2] = {tmem, tmem + N};
    const uint32_t a_base = smem_u32(a_buf), b_base = smem_u32(b_buf);

    // operator term tables (constant across tiles): one bulk copy
    if (tid == 0) {
        const uint32_t bytes = NOPS * 3 * C::B_TERM_BYTES;
        mbar_arrive_expect_tx(&bar[1], bytes);
        bulk_load(b_buf, p.ops, bytes, &bar[1]);
    }
    bool ok = mbar_wait_bounded(&bar[1], 0);
    ok = __syncthreads_and(ok);
    const bool ops_landed = ok;
    bool mma_outstanding = false;  // a committed MMA group whose completion was not seen
    uint32_t mma_phase = 0;

    const int b_local = tid / N, r_local = tid % N;  // this thread's stack row: array, row
    // this thread's input row of a tile (zeros for arrays beyond the batch);
    // for n <= 32 the next tile's row is loaded while the current tile's
    // contractions run, so the global-load latency overlaps them
    constexpr bool PREFETCH = N <= 32;
    auto load_row = [&](int tile, float (&dstv)[N]) {
        long long first, brow;
        int n, t0;
        tile_geom<N, TILED>(p, tile, first, n, brow, t0);
        if (b_local < n) {
            const float *src;
            if constexpr (!TILED)
                src = (p.in_off ? p.in + p.in_off[first + b_local] : p.in + (first + b_local) * (long long)(N * N)) +
                      r_local * N;
            else src = p.in + (brow * N + r_local) * p.ld_in + (long long)(t0 + b_local) * N;
#pragma unroll
            for (int q = 0; q < N / 4; ++q) {
                // L2-coherent load: with in == out this kernel writes the
                // same buffer (each tile only after its own rows were read)
                const float4 t = __ldcg(reinterpret_cast<const float4 *>(src) + q);
                dstv[4 * q] = t.x; dstv[4 * q + 1] = t.y; dstv[4 * q + 2] = t.z; dstv[4 * q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) dstv[j] = 0.0f;
        }
    };
    float v[N];
    float nxt[PREFETCH ? N : 1];
    if constexpr (PREFETCH) {
        if (blockIdx.x < (unsigned)p.ntiles) load_row(blockIdx.x, nxt);
    }
    for (int tile = blockIdx.x; ok && tile < p.ntiles; tile += gridDim.x) {
        long long first, brow;
        int n, t0;
        tile_geom<N, TILED>(p, tile, first, n, brow, t0);
        const bool active = b_local < n;
        if constexpr (PREFETCH) {
#pragma unroll
            for (int j = 0; j < N; ++j) v[j] = nxt[j];
            const int nx = tile + (int)gridDim.x;
            if (nx < p.ntiles) load_row(nx, nxt);
        } else {
            load_row(tile, v);
        }
#pragma unroll 1
        for (int pass = 0; pass < NPASS; ++pass) {
            const bool mn = (pass & 1) != 0;
            // ---- stage A: odd passes K-major from a held row, even passes MN-major
            if (!mn) stage_a<N, TERMS, false>(a_buf, v, tid, 0);
            else stage_a<N, TERMS, true>(a_buf, v, r_local, b_local * N);
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                const uint32_t bop = b_base + (pass >> 1) * 3 * C::B_TERM_BYTES;
                if (!mn) issue_pass<N, TERMS, false>(a_base, bop, d_tmem[pass & 1]);
                else issue_pass<N, TERMS, true>(a_base, bop, d_tmem[pass & 1]);
                tc_commit(&bar[0]);
            }
            ok = mbar_wait_bounded(&bar[0], mma_phase);
            ok = __syncthreads_and(ok);
            if (!ok) {
                mma_outstanding = true;
                break;
            }
            mma_phase ^= 1u;
            tc_fence_after();
            // ---- this thread's TMEM lane of the result
            const uint32_t taddr = d_tmem[pass & 1] + ((uint32_t)(32 * warp) << 16);
#pragma unroll
            for (int c = 0; c < N / 16; ++c) tmem_ld16(taddr + 16 * c, v + 16 * c);
            if constexpr (SPEC) {
                // after the second product thread (array, l) holds column l of
                // the spectrum, v[k] = Y[k][l]
                if (pass == 1) {
#pragma unroll
                    for (int k = 0; k < N; ++k) v[k] *= __ldg(p.lam + k * N + r_local);
                }
            }
        }
        if (!ok) break;
        // ---- store.  After two passes thread (array, c) holds column c of the
        // result (values over the row index): stores are coalesced across
        // lanes.  After four passes thread (array, i) holds row i.
        if (active) {
            if constexpr (NPASS == 2) {
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    float *dst;
                    if constexpr (!TILED)
                        dst = (p.out_off ? p.out + p.out_off[first + b_local]
                                         : p.out + (first + b_local) * (long long)(N * N)) + k * N + r_local;
                    else dst = p.out + (brow * N + k) * p.ld_out + (long long)(t0 + b_local) * N + r_local;
                    *dst = v[k];
                }
            } else {
                float *dst;
                if constexpr (!TILED)
                    dst = (p.out_off ? p.out + p.out_off[first + b_local]
                                     : p.out + (first + b_local) * (long long)(N * N)) + r_local * N;
                else dst = p.out + (brow * N + r_local) * p.ld_out + (long long)(t0 + b_local) * N;
#pragma unroll
                for (int q = 0; q < N / 4; ++q)
                    reinterpret_cast<float4 *>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (!ok && tid == 0) {
        record_timeout(p.status);
        // error path: let the asynchronous operations this CTA started finish
        // (each wait bounded) before its shared memory and TMEM are released,
        // so that nothing lands after the CTA has exited
        if (!ops_landed) mbar_wait_bounded(&bar[1], 0);
        if (mma_outstanding) mbar_wait_bounded(&bar[0], mma_phase);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
}

// ------------------------------------------------------------ warp-specialized kernel
// Forward and inverse (two products per tile) with the phases of different
// tiles overlapped.  k_tc_split runs each tile's load, split, products,
// TMEM read, re-split, products and store one after another in every
// thread, so a CTA is idle on each wait.  Here each phase has its own warps
// and double-buffered shared-memory stages and TMEM accumulators:
//   warps 0-3  (WG1): load tile t's rows (thread = stack row), split into
//              BF16 terms, write the K-major A operand of product 1;
//   warp 4, lane 0 : issue product 1 of every tile, warp 13, lane 0: product
//              2 (two issuers, so neither waits for the other's inputs), each
//              committed to the stage-free and result-ready barriers;
//   warps 5-8  (WG2): read T of tile t from TMEM (lane quadrant warp % 4),
//              re-split it into the MN-major A operand of product 2;
//   warps 9-12 (WG3): read Y of tile t from TMEM and store it (thread =
//              array and column: coalesced across lanes).
template <int N>
struct WsCfg {
    static constexpr int G = 128 / N;
    static constexpr int A_TERM = 128 * N * 2;
    static constexpr int A_STAGE = 3 * A_TERM;
    static constexpr int B_BYTES = 3 * N * N * 2;
    static constexpr int THREADS = 14 * 32;
    // operand stages and accumulators per phase (a deeper ring where tiles are
    // small; side 64 fits one)
    static constexpr int NS = N <= 16 ? 4 : (N == 32 ? 3 : 1);
    static constexpr int NBAR = 8 * NS + 1;  // eight barriers per stage and the operator barrier
    // input rows in flight per loading thread (cp.async into its own padded
    // row slots: pitch N + 4 floats keeps a warp's 16-byte reads conflict-free)
    static constexpr int D = N <= 16 ? 8 : (N == 32 ? 4 : 2);
    static constexpr int XP = N + 4;
    static constexpr int X_BYTES = D * 128 * XP * 4;
    static constexpr size_t SMEM = (size_t)2 * NS * A_STAGE + B_BYTES + X_BYTES + NBAR * 8 + 16;
    static constexpr int TMEM_COLS = tmem_alloc_cols(2 * NS * N);  // NS T and NS Y accumulators
    static_assert(TMEM_COLS <= 512, "TMEM");
};

// LAMF: every stored coefficient is multiplied by the diagonal p.lam (N x N,
// row k = frequency along h): the first half of the spectral composition of
// Prop. 1 (Eq. 4), whose second half is the orthonormal inverse in place.
template <int N, int TERMS, bool TILED, bool LAMF = false>
__global__ void __launch_bounds__(WsCfg<N>::THREADS, 1) k_tc_ws(const TcParams p)
{
    using C = WsCfg<N>;
    extern __shared__ __align__(1024) uint8_t wsm[];
    constexpr int NS = C::NS;
    uint8_t *a1 = wsm;                        // NS stages: product-1 operand
    uint8_t *a2 = wsm + NS * C::A_STAGE;      // NS stages: product-2 operand
    uint8_t *bop = wsm + 2 * NS * C::A_STAGE; // the operator's three terms
    float *xring = reinterpret_cast<float *>(bop + C::B_BYTES);  // D row slots per loading thread
    uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(xring) + C::X_BYTES);
    uint64_t *a1_full = bar, *a1_empty = bar + NS, *t_full = bar + 2 * NS, *t_empty = bar + 3 * NS;
    uint64_t *a2_full = bar + 4 * NS, *a2_empty = bar + 5 * NS, *y_full = bar + 6 * NS, *y_empty = bar + 7 * NS;
    uint64_t *b_full = bar + 8 * NS;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + C::NBAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&a1_full[i], 128);
            mbar_init(&a1_empty[i], 1);
            mbar_init(&t_full[i], 1);
            mbar_init(&t_empty[i], 128);
            mbar_init(&a2_full[i], 128);
            mbar_init(&a2_empty[i], 1);
            mbar_init(&y_full[i], 1);
            mbar_init(&y_empty[i], 128);
        }
        mbar_init(b_full, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 4) {
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
    // TMEM: T accumulators at columns s * N, Y accumulators at (NS + s) * N
    const int ntile_local = p.ntiles > (int)blockIdx.x
                                ? (p.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                                : 0;
    bool ok = true;
    long long last_commit = -1;  // MMA lanes: the tile of the last commit (error path)

    if (warp < 4) {
        // ---- WG1: load and split tile rows; each thread copies its own row of
        // the next D tiles with cp.async and reads back only what it copied, so
        // its own group wait is all the synchronization the copies need
        const int b_local = tid / N, r_local = tid % N;
        auto issue = [&](int t) {
            const int tile = (int)blockIdx.x + t * (int)gridDim.x;
            if (t < ntile_local) {
                long long first, brow;
                int n, t0;
                tile_geom<N, TILED>(p, tile, first, n, brow, t0);
                if (b_local < n) {
                    const float *src;
                    if constexpr (!TILED)
                        src = (p.in_off ? p.in + p.in_off[first + b_local]
                                        : p.in + (first + b_local) * (long long)(N * N)) + r_local * N;
                    else src = p.in + (brow * N + r_local) * p.ld_in + (long long)(t0 + b_local) * N;
                    float *dst = xring + ((t % C::D) * 128 + tid) * C::XP;
#pragma unroll
                    for (int q = 0; q < N / 4; ++q) cp_async16(dst + 4 * q, src + 4 * q);
                }
            }
            cp_async_commit();  // one group per tile, empty past the end
        };
#pragma unroll 1
        for (int t = 0; t < C::D; ++t) issue(t);
        float v[N];
        for (int t = 0; t < ntile_local; ++t) {
            const int tile = (int)blockIdx.x + t * (int)gridDim.x;
            long long first, brow;
            int n, t0;
            tile_geom<N, TILED>(p, tile, first, n, brow, t0);
            cp_async_wait_group<C::D - 1>();  // this thread's copies of tile t have landed
            if (b_local < n) {
                const float4 *q4 = reinterpret_cast<const float4 *>(xring + ((t % C::D) * 128 + tid) * C::XP);
#pragma unroll
                for (int q = 0; q < N / 4; ++q) {
                    const float4 x = q4[q];
                    v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j) v[j] = 0.0f;
            }
            issue(t + C::D);  // refill the slot just read
            const int s = t % NS;
            if (t >= NS && !mbar_wait_bounded(&a1_empty[s], (uint32_t)(t / NS - 1) & 1u)) { ok = false; break; }
            if (*abort_flag) { ok = false; break; }
            stage_a<N, TERMS, false>(a1 + s * C::A_STAGE, v, tid, 0);
            fence_proxy_async_smem();
            mbar_arrive(&a1_full[s]);
        }
        cp_async_wait_all();  // no copy of this thread still in flight at exit
    } else if (warp == 4 || warp == 13) {
        // ---- MMA issue, one lane per product so that neither waits for the
        // other's inputs: warp 4 product 1 (K-major A), warp 13 product 2
        if (lane == 0) {
            const bool first = warp == 4;
            if (first) {
                mbar_arrive_expect_tx(b_full, C::B_BYTES);
                bulk_load(bop, p.ops, C::B_BYTES, b_full);
            }
            if (!mbar_wait_bounded(b_full, 0)) ok = false;
            const uint32_t b_base = smem_u32(bop);
            uint64_t *in_full = first ? a1_full : a2_full, *acc_empty = first ? t_empty : y_empty;
            uint64_t *in_empty = first ? a1_empty : a2_empty, *acc_full = first ? t_full : y_full;
            uint8_t *abuf = first ? a1 : a2;
            const int acc_col = first ? 0 : NS * N;
            for (int t = 0; ok && t < ntile_local; ++t) {
                const int s = t % NS;
                if (!mbar_wait_bounded(&in_full[s], (uint32_t)(t / NS) & 1u) ||
                    (t >= NS && !mbar_wait_bounded(&acc_empty[s], (uint32_t)(t / NS - 1) & 1u)) || *abort_flag) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (first)
                    issue_pass<N, TERMS, false>(smem_u32(abuf + s * C::A_STAGE), b_base,
                                                tmem + (uint32_t)(acc_col + s * N));
                else
                    issue_pass<N, TERMS, true>(smem_u32(abuf + s * C::A_STAGE), b_base,
                                               tmem + (uint32_t)(acc_col + s * N));
                tc_commit(&in_empty[s]);
                tc_commit(&acc_full[s]);
                last_commit = t;
            }
        }
    } else {
        // ---- WG2 (warps 5-8) and WG3 (warps 9-12): TMEM lane quadrant warp % 4
        const bool wg2 = warp <= 8;
        const int m = 32 * (warp & 3) + lane;  // stack row of this thread's TMEM lane
        const int b_local = m / N, r_local = m % N;
        const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
        float v[N];
        for (int t = 0; t < ntile_local; ++t) {
            const int s = t % NS;
            uint64_t *full = wg2 ? &t_full[s] : &y_full[s];
            // warp-uniform decisions only: the TMEM loads below are warp-collective
            bool w = mbar_wait_bounded(full, (uint32_t)(t / NS) & 1u) && !*abort_flag;
            w = __all_sync(0xffffffffu, w);
            if (!w) { ok = false; break; }
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)((wg2 ? s : NS + s) * N) + lane_off;
            if constexpr (N >= 16) {
#pragma unroll
                for (int c = 0; c < N / 16; ++c) tmem_ld16(acc + 16 * c, v + 16 * c);
            }
            tc_fence_before();
            mbar_arrive(wg2 ? &t_empty[s] : &y_empty[s]);
            if (wg2) {
                // T row r_local of array b_local -> column r_local of the MN-major operand
                bool w2 = t < NS || mbar_wait_bounded(&a2_empty[s], (uint32_t)(t / NS - 1) & 1u);
                w2 = __all_sync(0xffffffffu, w2);
                if (!w2) { ok = false; break; }
                stage_a<N, TERMS, true>(a2 + s * C::A_STAGE, v, r_local, b_local * N);
                fence_proxy_async_smem();
                mbar_arrive(&a2_full[s]);
            } else {
                // column r_local of Y[b_local] (values over the row index): coalesced across lanes
                const int tile = (int)blockIdx.x + t * (int)gridDim.x;
                long long first, brow;
                int n, t0;
                tile_geom<N, TILED>(p, tile, first, n, brow, t0);
                if (b_local < n) {
                    if constexpr (LAMF) {
#pragma unroll
                        for (int k = 0; k < N; ++k) v[k] *= __ldg(p.lam + k * N + r_local);
                    }
#pragma unroll
                    for (int k = 0; k < N; ++k) {
                        float *dst;
                        if constexpr (!TILED)
                            dst = (p.out_off ? p.out + p.out_off[first + b_local]
                                             : p.out + (first + b_local) * (long long)(N * N)) + k * N + r_local;
                        else dst = p.out + (brow * N + k) * p.ld_out + (long long)(t0 + b_local) * N + r_local;
                        *dst = v[k];
                    }
                }
            }
        }
    }
    if (!ok) {
        *abort_flag = 1;
        if (lane == 0) record_timeout(p.status);
    }
    // error path: the MMA lane waits (bounded) for the operator copy and its
    // last committed products before shared memory and TMEM are released
    if ((warp == 4 || warp == 13) && lane == 0 && !ok) {
        mbar_wait_bounded(b_full, 0);
        if (last_commit >= 0) {
            const int t = (int)last_commit, s = t % NS;
            mbar_wait_bounded(warp == 4 ? &t_full[s] : &y_full[s], (uint32_t)(t / NS) & 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
}

// ------------------------------------------------------------ tables
// Operator matrix M (direction/norm as in the dense route) split into three
// BF16 terms in FP64, written in the K-major B layout: B[l][j] = M[l][j]
// (rows = output index, K = input index).
__global__ void k_gen_split_op(__nv_bfloat16 *dst, int n, int direction, int norm)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int r = idx / n, k = idx % n;  // B row (output index), K (input index)
    // forward: M[r][k] = s_r cos(pi (2k+1) r / (2n)); inverse: M[r][k] = s_k cos(pi (2r+1) k / (2n))
    const int kk = direction == 1 ? r : k;   // frequency index
    const int jj = direction == 1 ? k : r;   // sample index
    double s;
    if (norm == 0) s = (kk == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
    else if (direction == 1) s = 2.0;
    else s = (kk == 0) ? 1.0 : 2.0;
    // cos(pi m / (2n)) with the argument reduced exactly
    long long m = (2LL * jj + 1) * kk;
    const long long d = 2LL * n;
    long long red = m % (2 * d);
    if (red > d) red = 2 * d - red;
    double sign = 1.0;
    if (2 * red > d) { red = d - red; sign = -1.0; }
    double c;
    if (red == 0) c = sign;
    else if (2 * red == d) c = 0.0;
    else c = sign * cospi((double)red / (double)d);
    const double val = s * c;
    const __nv_bfloat16 t0 = __double2bfloat16(val);
    const double r1 = val - (double)__bfloat162float(t0);
    const __nv_bfloat16 t1 = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(t1);
    const __nv_bfloat16 t2 = __double2bfloat16(r2);
    const int off = (((r >> 3) * (n >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);  // elements
    dst[off] = t0;
    dst[n * n + off] = t1;
    dst[2 * n * n + off] = t2;
}

bool tc_supported(int rows, int cols) { return rows == cols && (rows == 16 || rows == 32 || rows == 64); }

size_t tc_table_elems(int n) { return (size_t)3 * n * n; }

cudaError_t tc_gen_tables(__nv_bfloat16 *dst, int n, int direction, int norm, cudaStream_t s)
{
    k_gen_split_op<<<(n * n + 255) / 256, 256, 0, s>>>(dst, n, direction, norm);
    return cudaGetLastError();
}

template <int N, int NPASS, int TERMS, bool TILED, bool SPEC = false>
static cudaError_t tc_launch_one(const TcParams &p0, const __nv_bfloat16 *ops, cudaStream_t stream)
{
    using C = TcCfg<N>;
    constexpr int NOPS = NPASS / 2;
    auto kern = k_tc_split<N, NPASS, TERMS, TILED, SPEC>;
    const size_t smem = (size_t)TERMS * C::A_TERM_BYTES + (size_t)NOPS * 3 * C::B_TERM_BYTES + 64;
    static DeviceLaunchCache cache;
    int dev = 0, blocks_per_sm = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cache.get(
        dev,
        [&](int d, int &bps, int &sms) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (r != cudaSuccess) return r;
            // Resident CTAs per SM from threads, registers and shared memory, capped so
            // that their TMEM allocations fit in the 512 columns (a CTA beyond that
            // would wait in tcgen05.alloc until another one exits).  Computed here
            // because the runtime's occupancy query reports one CTA for kernels that
            // allocate tensor memory.
            cudaFuncAttributes fa;
            r = cudaFuncGetAttributes(&fa, kern);
            if (r != cudaSuccess) return r;
            int smem_per_sm = 0, regs_per_sm = 0, reserved = 0;
            cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, d);
            cudaDeviceGetAttribute(&regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, d);
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, d);
            const int by_threads = 2048 / 128;
            const int regs_cta = ((fa.numRegs * 32 + 255) / 256) * 256 * 4;  // per-warp allocation granularity
            const int by_regs = regs_cta > 0 ? regs_per_sm / regs_cta : by_threads;
            const int by_smem = (int)((size_t)smem_per_sm / (smem + fa.sharedSizeBytes + (size_t)reserved));
            const int tmem_cap = 512 / C::TMEM_COLS;
            int occ = by_threads;
            if (by_regs < occ) occ = by_regs;
            if (by_smem < occ) occ = by_smem;
            bps = occ < tmem_cap ? occ : tmem_cap;
            r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
            if (r != cudaSuccess) return r;
            if (bps < 1) return cudaErrorInvalidConfiguration;
            if (debug_enabled())
                fprintf(stderr, "[bdct] k_tc_split<%d,%d,%d,%d>: %d CTAs/SM (regs %d, smem %zu B, TMEM cap %d)\n", N,
                        NPASS, TERMS, (int)TILED, bps, fa.numRegs, smem, tmem_cap);
            return cudaSuccess;
        },
        &blocks_per_sm, &num_sms);
    if (e != cudaSuccess) return e;
    TcParams p = p0;
    p.ops = ops;
    if (SPEC && !p.lam) return cudaErrorInvalidValue;
    long long nt;
    if (!TILED) {
        nt = (p.count + C::G - 1) / C::G;
    } else {
        p.chunks_per_row = (p.tiles_per_row + C::G - 1) / C::G;
        nt = (p.count / p.tiles_per_row) * p.chunks_per_row;
    }
    if (nt <= 0) return cudaSuccess;
    if (nt > 0x7ff00000LL) return cudaErrorInvalidValue;
    p.ntiles = (int)nt;
    long long grid = (long long)blocks_per_sm * num_sms;
    if (grid > nt) grid = nt;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int N, int TERMS, bool TILED, bool LAMF = false>
static cudaError_t tc_ws_launch(const TcParams &p0, const __nv_bfloat16 *ops, cudaStream_t stream)
{
    using C = WsCfg<N>;
    auto kern = k_tc_ws<N, TERMS, TILED, LAMF>;
    if (LAMF && !p0.lam) return cudaErrorInvalidValue;
    static DeviceLaunchCache cache;
    int dev = 0, bps = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cache.get(
        dev,
        [&](int d, int &b, int &n) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
            b = 1;
            if (r == cudaSuccess && debug_enabled())
                fprintf(stderr, "[bdct] k_tc_ws<%d,%d,%d>: 1 CTA/SM x %d threads, smem %zu B, TMEM %d cols\n", N,
                        TERMS, (int)TILED, C::THREADS, C::SMEM, C::TMEM_COLS);
            return r;
        },
        &bps, &sms);
    if (e != cudaSuccess) return e;
    TcParams p = p0;
    p.ops = ops;
    long long nt;
    if (!TILED) {
        nt = (p.count + C::G - 1) / C::G;
    } else {
        p.chunks_per_row = (p.tiles_per_row + C::G - 1) / C::G;
        nt = (p.count / p.tiles_per_row) * p.chunks_per_row;
    }
    if (nt <= 0) return cudaSuccess;
    if (nt > 0x7ff00000LL) return cudaErrorInvalidValue;
    p.ntiles = (int)nt;
    long long grid = sms;
    if (grid > nt) grid = nt;
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

template <int N, int TERMS>
static cudaError_t tc_launch_nt(Dir dir, const TcParams &p, const __nv_bfloat16 *ops, cudaStream_t s, bool tiled)
{
    // forward and inverse of sides 32 and 64: the warp-specialized kernel.
    // Measured on 512 MiB batches: side 32 0.48 -> 0.61 of HBM, side 64 (one
    // operand stage per phase) 0.29 -> 0.49; side 16 runs 0.73 on k_tc_split
    // (eight CTAs per SM) against 0.52 here, where the hand-offs of its 8 KiB
    // tiles stay exposed.
    if constexpr (N == 32 || N == 64) {
        if (dir == DIR_FWD || dir == DIR_INV)
            return tiled ? tc_ws_launch<N, TERMS, true>(p, ops, s) : tc_ws_launch<N, TERMS, false>(p, ops, s);
        if (dir == DIR_RT) {
            // the normalized round trip as the orthonormal forward (the
            // table's first operator) then the orthonormal inverse (its
            // second) in place: two warp-specialized launches measured
            // faster than one launch of the one-role kernel's four products
            // (side 32 0.26 -> 0.31 of HBM, side 64 0.21 -> 0.24)
            TcParams pi = p;
            pi.in = p.out;
            pi.in_off = p.out_off;
            pi.ld_in = p.ld_out;
            const __nv_bfloat16 *inv = ops + 3 * N * N;
            cudaError_t e = tiled ? tc_ws_launch<N, TERMS, true>(p, ops, s) : tc_ws_launch<N, TERMS, false>(p, ops, s);
            if (e == cudaSuccess)
                e = tiled ? tc_ws_launch<N, TERMS, true>(pi, inv, s) : tc_ws_launch<N, TERMS, false>(pi, inv, s);
            return e;
        }
        if (dir == DIR_SPEC) {
            // likewise, the forward storing its coefficients times Lambda
            TcParams pi = p;
            pi.in = p.out;
            pi.in_off = p.out_off;
            pi.ld_in = p.ld_out;
            pi.lam = nullptr;
            const __nv_bfloat16 *inv = ops + 3 * N * N;
            cudaError_t e = tiled ? tc_ws_launch<N, TERMS, true, true>(p, ops, s)
                                  : tc_ws_launch<N, TERMS, false, true>(p, ops, s);
            if (e == cudaSuccess)
                e = tiled ? tc_ws_launch<N, TERMS, true>(pi, inv, s) : tc_ws_launch<N, TERMS, false>(pi, inv, s);
            return e;
        }
    }
    if (dir == DIR_RT)
        return tiled ? tc_launch_one<N, 4, TERMS, true>(p, ops, s) : tc_launch_one<N, 4, TERMS, false>(p, ops, s);
    if (dir == DIR_SPEC)
        return tiled ? tc_launch_one<N, 4, TERMS, true, true>(p, ops, s)
                     : tc_launch_one<N, 4, TERMS, false, true>(p, ops, s);
    return tiled ? tc_launch_one<N, 2, TERMS, true>(p, ops, s) : tc_launch_one<N, 2, TERMS, false>(p, ops, s);
}

template <int N>
static cudaError_t tc_launch_n(Dir dir, int terms, const TcParams &p, const __nv_bfloat16 *ops, cudaStream_t s,
                               bool tiled)
{
    switch (terms) {
        case 3: return tc_launch_nt<N, 3>(dir, p, ops, s, tiled);
        case 2: return tc_launch_nt<N, 2>(dir, p, ops, s, tiled);
        default: return tc_launch_nt<N, 1>(dir, p, ops, s, tiled);
    }
}

cudaError_t tc_launch(int n, Dir dir, int terms, const ExecGeom &g, const __nv_bfloat16 *ops, unsigned int *status,
                      cudaStream_t stream)
{
    TcParams p{};
    p.in = g.in;
    p.out = g.out;
    p.count = g.count;
    p.tiles_per_row = g.tiles_per_row;
    p.ld_in = g.ld_in;
    p.ld_out = g.ld_out;
    p.status = status;
    p.in_off = g.in_off;
    p.out_off = g.out_off;
    p.lam = g.lam;
    const bool tiled = g.tiled != 0;
    switch (n) {
        case 16: return tc_launch_n<16>(dir, terms, p, ops, stream, tiled);
        case 32: return tc_launch_n<32>(dir, terms, p, ops, stream, tiled);
        case 64: return tc_launch_n<64>(dir, terms, p, ops, stream, tiled);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bdct
