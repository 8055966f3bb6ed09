// C ABI: plans, argument validation and dispatch to the kernel families.
//
// A plan (Section 3.2 of the BRiDCT paper: plan-owned tables and workspace,
// no allocation or planning inside a transform) fixes the shape, the
// directions served, the normalization and the path.  Execution calls only
// validate pointers and launch kernels on the caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "bdct_internal.h"
#include "plan.h"
#include "small_dense.h"
#include "fp32_ring.h"
#include "fp32_lines.h"
#include "dense_passes.h"

using namespace bdct;

namespace {

thread_local int t_last_cuda_error = 0;

int cuda_fail(cudaError_t e)
{
    t_last_cuda_error = (int)e;
    return BDCT_ERR_CUDA;
}

// Workspace of the separable routes: arrays per chunk are chosen so that a
// chunk holds at least one array and about 256 MiB.  Every chunk costs two
// pass launches with their ramp-up and drain: measured on 256^2 batches
// 0.30 / 0.34 / 0.35 of HBM with 64 / 128 / 256 MiB chunks, 768 x 1024
// batches 0.23 / 0.26 / 0.28 (bdct_plan_set_chunk_bytes changes it per plan).
constexpr size_t kChunkBytes = 256ull << 20;

}  // namespace

static AxisScale axis_scale(int n, Dir dir, int norm)
{
    const double a0 = std::sqrt(1.0 / n), a1 = std::sqrt(2.0 / n);
    switch (dir) {
        case DIR_FWD:
            if (norm == BDCT_NORM_ORTHO) return {(float)a0, (float)a1};
            return {2.0f, 2.0f};
        case DIR_INV:
            if (norm == BDCT_NORM_ORTHO) return {(float)a0, (float)a1};
            return {1.0f, 2.0f};
        default:  // E_n^2 between the forward core and its adjoint (Prop. 1)
            return {(float)(1.0 / n), (float)(2.0 / n)};
    }
}

static int check_device(int *dev_out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    int major = 0, minor = 0;
    e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (major != 10 || minor != 3) return BDCT_ERR_ARCH;
    *dev_out = dev;
    return BDCT_OK;
}

static void plan_free(bdct_plan *p)
{
    if (!p) return;
    if (p->ops) cudaFree(p->ops);
    if (p->status) cudaFree(p->status);
    if (p->tc_ops) cudaFree(p->tc_ops);
    if (p->tg_ops) cudaFree(p->tg_ops);
    if (p->tg_abuf) cudaFree(p->tg_abuf);
    if (p->line_tw) cudaFree(p->line_tw);
    if (p->spec_plain) cudaFree(p->spec_plain);
    if (p->spec_fold) cudaFree(p->spec_fold);
    if (p->rp_bits) cudaFree(p->rp_bits);
    host_staging_free(p);
    if (p->work) cudaFree(p->work);
    delete p;
}

// Shapes of the tensor-core separable passes: both sides 16, 32 or a multiple
// of 64 (up to 8192), or 8 x 8 through the Kronecker operator.
static bool tg_supported(int rows, int cols)
{
    return (rows == 8 && cols == 8) || (tg_axis_ok(rows) && tg_axis_ok(cols));
}

// Build the blocked operator tables of a variant-4 plan: one per distinct
// (side, direction, normalization) among the slots the plan's kinds need.
static int tg_plan_tables(bdct_plan *p)
{
    struct Want { int slot, axis, n, direction, norm; };
    Want want[8];
    int nw = 0;
    const unsigned k = p->kind;
    const bool pair = (k & (BDCT_ROUNDTRIP | BDCT_SPECTRAL)) != 0;
    auto add = [&](int slot, int direction, int norm) {
        if (p->tg_kron) {
            want[nw++] = Want{slot, 0, 8, direction, norm};
        } else {
            want[nw++] = Want{slot, 0, p->rows, direction, norm};
            want[nw++] = Want{slot, 1, p->cols, direction, norm};
        }
    };
    if (k & BDCT_FORWARD) add(0, 1, p->norm);
    if (k & BDCT_INVERSE) add(1, 2, p->norm);
    if (pair) { add(2, 1, BDCT_NORM_ORTHO); add(3, 2, BDCT_NORM_ORTHO); }
    // distinct tables, each 3 n^2 BF16 elements (64 x 64 for the Kronecker operator)
    int uniq[8][3];
    size_t uoff[8];
    int nu = 0;
    size_t total = 0;
    size_t off_of[8];
    for (int i = 0; i < nw; ++i) {
        int j = 0;
        for (; j < nu; ++j)
            if (uniq[j][0] == want[i].n && uniq[j][1] == want[i].direction && uniq[j][2] == want[i].norm) break;
        if (j == nu) {
            uniq[nu][0] = want[i].n; uniq[nu][1] = want[i].direction; uniq[nu][2] = want[i].norm;
            uoff[nu] = total;
            total += tg_table_elems(p->tg_kron ? 64 : want[i].n);
            ++nu;
        }
        off_of[i] = uoff[j];
    }
    cudaError_t e = cudaMalloc(&p->tg_ops, total * sizeof(__nv_bfloat16));
    if (e != cudaSuccess) { t_last_cuda_error = (int)e; return BDCT_ERR_NO_MEMORY; }
    p->table_bytes = total * sizeof(__nv_bfloat16);
    for (int j = 0; j < nu && e == cudaSuccess; ++j)
        e = tg_gen_table(p->tg_ops + uoff[j], uniq[j][0], uniq[j][1], uniq[j][2], p->tg_kron, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < nw; ++i) {
        if (want[i].axis == 0) p->tg_h[want[i].slot] = off_of[i];
        else p->tg_w[want[i].slot] = off_of[i];
    }
    return BDCT_OK;
}

// The input-term buffer of the warp-specialized tensor-core passes (long
// contractions): three BF16 terms of every element of a chunk, in whole
// 128-row tiles, for either pass.  Only plans with such an axis get one.
static cudaError_t tg_alloc_split(bdct_plan *p)
{
    if (p->tg_abuf) { cudaFree(p->tg_abuf); p->tg_abuf = nullptr; }
    if (p->tg_kron) return cudaSuccess;
    const long long nb = p->chunk_arrays;
    const size_t e1 = tg_split_elems(nb * p->rows, p->cols), e2 = tg_split_elems(nb * p->cols, p->rows);
    const size_t elems = e1 > e2 ? e1 : e2;
    if (p->rows % 128 && p->cols % 128) return cudaSuccess;  // no axis on the long-contraction kernel
    return cudaMalloc(&p->tg_abuf, elems * sizeof(__nv_bfloat16));
}

extern "C" int bdct_plan_create(bdct_plan **plan, int rows, int cols, unsigned kind, int norm, int path)
{
    if (!plan) return BDCT_ERR_INVALID_ARG;
    *plan = nullptr;
    if (rows < 1 || cols < 1) return BDCT_ERR_INVALID_ARG;
    if (kind == 0 || (kind & ~(BDCT_FORWARD | BDCT_INVERSE | BDCT_ROUNDTRIP | BDCT_SPECTRAL)))
        return BDCT_ERR_INVALID_ARG;
    if (norm != BDCT_NORM_ORTHO && norm != BDCT_NORM_NONE) return BDCT_ERR_INVALID_ARG;
    if (path < BDCT_PATH_AUTO || path > BDCT_PATH_BF16) return BDCT_ERR_INVALID_ARG;
    if (rows > 8192 || cols > 8192) return BDCT_ERR_UNSUPPORTED_SHAPE;
    if (cols % 4 != 0) return BDCT_ERR_UNSUPPORTED_SHAPE;

    int dev = 0;
    int st = check_device(&dev);
    if (st != BDCT_OK) return st;

    int resolved = path;
    if (resolved == BDCT_PATH_AUTO) {
        // fused FP32 where it exists, else the tensor-core route, else dense passes
        if (fused_supported(rows, cols)) resolved = BDCT_PATH_FP32;
        else if (tc_supported(rows, cols)) resolved = BDCT_PATH_SPLIT_TC;
        else resolved = BDCT_PATH_FP32;
    }
    const bool tc_path = resolved == BDCT_PATH_SPLIT_TC || resolved == BDCT_PATH_SPLIT_HILO || resolved == BDCT_PATH_BF16;
    // tensor cores: on chip for squares 16..64, separable passes for the rest
    const bool tc = tc_path && tc_supported(rows, cols);
    const bool tg = tc_path && !tc && tg_supported(rows, cols);
    if (tc_path && !tc && !tg) return BDCT_ERR_UNSUPPORTED_SHAPE;

    bdct_plan *p = new (std::nothrow) bdct_plan;
    if (!p) return BDCT_ERR_NO_MEMORY;
    p->rows = rows;
    p->cols = cols;
    p->kind = kind;
    p->norm = norm;
    p->path = resolved;
    p->device = dev;
    for (int d = 0; d < 3; ++d) {
        p->scales[d].h = axis_scale(rows, (Dir)d, norm);
        p->scales[d].w = axis_scale(cols, (Dir)d, norm);
    }

    cudaError_t e = fused_init_device(dev);
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e); }
    e = cudaMalloc(&p->status, sizeof(unsigned int));
    if (e != cudaSuccess) { plan_free(p); t_last_cuda_error = (int)e; return BDCT_ERR_NO_MEMORY; }
    e = cudaMemset(p->status, 0, sizeof(unsigned int));
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e); }

    if (tc) {
        p->variant = 3;
        p->tc_terms = resolved == BDCT_PATH_SPLIT_TC ? 3 : (resolved == BDCT_PATH_SPLIT_HILO ? 2 : 1);
        const size_t te = tc_table_elems(rows);
        // the round trip and the spectral direction share the orthonormal pair
        const bool pair = (kind & (BDCT_ROUNDTRIP | BDCT_SPECTRAL)) != 0;
        const size_t ntab = ((kind & BDCT_FORWARD) ? 1 : 0) + ((kind & BDCT_INVERSE) ? 1 : 0) + (pair ? 2 : 0);
        e = cudaMalloc(&p->tc_ops, ntab * te * sizeof(__nv_bfloat16));
        if (e != cudaSuccess) { plan_free(p); t_last_cuda_error = (int)e; return BDCT_ERR_NO_MEMORY; }
        p->table_bytes = ntab * te * sizeof(__nv_bfloat16);
        size_t off = 0;
        if (kind & BDCT_FORWARD) {
            p->tc_off[DIR_FWD] = off;
            e = tc_gen_tables(p->tc_ops + off, rows, 1, norm, 0);
            off += te;
        }
        if (e == cudaSuccess && (kind & BDCT_INVERSE)) {
            p->tc_off[DIR_INV] = off;
            e = tc_gen_tables(p->tc_ops + off, rows, 2, norm, 0);
            off += te;
        }
        if (e == cudaSuccess && pair) {
            // the round trip is normalized: orthonormal forward, then its adjoint
            p->tc_off[DIR_RT] = off;
            e = tc_gen_tables(p->tc_ops + off, rows, 1, BDCT_NORM_ORTHO, 0);
            if (e == cudaSuccess) e = tc_gen_tables(p->tc_ops + off + te, rows, 2, BDCT_NORM_ORTHO, 0);
            off += 2 * te;
        }
        if (e != cudaSuccess) { plan_free(p); return cuda_fail(e); }
    } else if (tg) {
        p->variant = 4;
        p->tc_terms = resolved == BDCT_PATH_SPLIT_TC ? 3 : (resolved == BDCT_PATH_SPLIT_HILO ? 2 : 1);
        p->tg_kron = rows == 8 && cols == 8;
        st = tg_plan_tables(p);
        if (st != BDCT_OK) { plan_free(p); return st; }
        // workspace: whole arrays, about kChunkBytes per chunk
        const size_t arr_bytes = (size_t)rows * cols * sizeof(float);
        long long chunk = (long long)(kChunkBytes / arr_bytes);
        if (chunk < 1) chunk = 1;
        p->chunk_arrays = chunk;
        p->work_bytes = (size_t)chunk * arr_bytes;
        e = cudaMalloc(&p->work, p->work_bytes);
        if (e != cudaSuccess) { plan_free(p); t_last_cuda_error = (int)e; return BDCT_ERR_NO_MEMORY; }
        e = tg_alloc_split(p);
        if (e != cudaSuccess) { plan_free(p); t_last_cuda_error = (int)e; return BDCT_ERR_NO_MEMORY; }
    } else if (fused_supported(rows, cols)) {
        p->variant = 1;
    } else if (lines_supported(rows) && lines_supported(cols)) {
        // two FFT line passes through the workspace, each writing transposed
        p->variant = 2;
        p->lines = true;
        const size_t arr_bytes = (size_t)rows * cols * sizeof(float);
        long long chunk = (long long)(kChunkBytes / arr_bytes);
        if (chunk < 1) chunk = 1;
        p->chunk_arrays = chunk;
        p->work_bytes = (size_t)chunk * arr_bytes;
        e = cudaMalloc(&p->work, p->work_bytes);
        if (e != cudaSuccess) { plan_free(p); t_last_cuda_error = (int)e; return BDCT_ERR_NO_MEMORY; }
        p->line_tw_h = lines_table_elems(cols);
        e = cudaMalloc(&p->line_tw, (lines_table_elems(cols) + lines_table_elems(rows)) * sizeof(float2));
        if (e != cudaSuccess) { plan_free(p); t_last_cuda_error = (int)e; return BDCT_ERR_NO_MEMORY; }
        e = lines_gen_table(p->line_tw, cols, 0);
        if (e == cudaSuccess) e = lines_gen_table(p->line_tw + p->line_tw_h, rows, 0);
        if (e != cudaSuccess) { plan_free(p); return cuda_fail(e); }
        p->table_bytes = (lines_table_elems(cols) + lines_table_elems(rows)) * sizeof(float2);
    } else {
        p->variant = 2;
        // operator matrices: forward and inverse in the plan's norm, and the
        // orthonormal pair for the round trip (which is normalized for both)
        size_t per_dir = (size_t)rows * rows + (size_t)cols * cols;
        size_t total = 0;
        const bool need[3] = {(kind & BDCT_FORWARD) != 0, (kind & BDCT_INVERSE) != 0,
                              (kind & (BDCT_ROUNDTRIP | BDCT_SPECTRAL)) != 0};
        size_t nmats = (need[0] ? 1 : 0) + (need[1] ? 1 : 0) + (need[2] ? 2 : 0);
        total = nmats * per_dir;
        e = cudaMalloc(&p->ops, total * sizeof(float));
        if (e != cudaSuccess) { plan_free(p); t_last_cuda_error = (int)e; return BDCT_ERR_NO_MEMORY; }
        p->table_bytes = total * sizeof(float);
        size_t off = 0;
        auto gen = [&](int direction, int nrm, size_t &oh, size_t &ow) -> cudaError_t {
            oh = off; off += (size_t)rows * rows;
            ow = off; off += (size_t)cols * cols;
            cudaError_t r = dense_gen_operator(p->ops + oh, rows, direction, nrm, 0);
            if (r == cudaSuccess) r = dense_gen_operator(p->ops + ow, cols, direction, nrm, 0);
            return r;
        };
        if (need[0] && e == cudaSuccess) e = gen(1, norm, p->op_h_off[DIR_FWD], p->op_w_off[DIR_FWD]);
        if (need[1] && e == cudaSuccess) e = gen(2, norm, p->op_h_off[DIR_INV], p->op_w_off[DIR_INV]);
        if (need[2] && e == cudaSuccess) {
            // RT forward half uses slot DIR_RT; its inverse half follows it
            size_t fh, fw, ih, iw;
            e = gen(1, BDCT_NORM_ORTHO, fh, fw);
            if (e == cudaSuccess) e = gen(2, BDCT_NORM_ORTHO, ih, iw);
            p->op_h_off[DIR_RT] = fh;
            p->op_w_off[DIR_RT] = fw;
            (void)ih; (void)iw;  // located at fh + per_dir
        }
        if (e != cudaSuccess) { plan_free(p); return cuda_fail(e); }
        if (small_dense_supported(rows, cols)) {
            // every pass in shared memory (small_dense.cu): no workspace
            p->small = true;
        } else {
            const size_t arr_bytes = (size_t)rows * cols * sizeof(float);
            long long chunk = (long long)(kChunkBytes / arr_bytes);
            if (chunk < 1) chunk = 1;
            p->chunk_arrays = chunk;
            const int nbuf = (kind & (BDCT_ROUNDTRIP | BDCT_SPECTRAL)) ? 2 : 1;
            p->work_bytes = (size_t)chunk * arr_bytes * nbuf;
            e = cudaMalloc(&p->work, p->work_bytes);
            if (e != cudaSuccess) { plan_free(p); t_last_cuda_error = (int)e; return BDCT_ERR_NO_MEMORY; }
        }
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { plan_free(p); return cuda_fail(e); }
    *plan = p;
    return BDCT_OK;
}

extern "C" int bdct_plan_destroy(bdct_plan *plan)
{
    if (!plan) return BDCT_OK;
    const int dev = plan->device;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    plan_free(plan);
    if (cur >= 0 && cur != dev) cudaSetDevice(cur);
    return BDCT_OK;
}

static int dir_of(unsigned kind, Dir *d)
{
    switch (kind) {
        case BDCT_FORWARD: *d = DIR_FWD; return BDCT_OK;
        case BDCT_INVERSE: *d = DIR_INV; return BDCT_OK;
        case BDCT_ROUNDTRIP: *d = DIR_RT; return BDCT_OK;
        case BDCT_SPECTRAL: *d = DIR_SPEC; return BDCT_OK;
        default: return BDCT_ERR_INVALID_ARG;
    }
}

static bool ranges_partially_overlap(const void *a, const void *b, size_t bytes)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    if (x == y) return false;
    return x < y + bytes && y < x + bytes;
}

static int run_lines(const bdct_plan *p, Dir dir, const DirScales &sc, const float *in, const long long *in_off,
                     float *out, const long long *out_off, long long count, cudaStream_t s,
                     const float *lam = nullptr)
{
    const int h = p->rows, w = p->cols;
    const long long hw = (long long)h * w;
    for (long long b0 = 0; b0 < count; b0 += p->chunk_arrays) {
        const long long nb = (count - b0) < p->chunk_arrays ? (count - b0) : p->chunk_arrays;
        const float *src = in_off ? in : in + b0 * hw;
        float *dst = out_off ? out : out + b0 * hw;
        // rows of X (h lines of w) -> workspace (w x h), then rows of that (w lines of h) -> out (h x w)
        cudaError_t e = lines_pass(src, p->work, h, w, nb, dir, sc.w, p->line_tw, p->status, s,
                                   in_off ? in_off + b0 : nullptr, nullptr);
        if (e == cudaSuccess)
            e = lines_pass_lam(p->work, dst, w, h, nb, dir, sc.h, p->line_tw + p->line_tw_h, p->status, s,
                               nullptr, out_off ? out_off + b0 : nullptr, true, lam);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return BDCT_OK;
}

// The dense route in shared memory (both sides at most 64): rows then
// columns (forward, inverse), and for the round trip and the spectral
// direction the adjoint columns then rows after them, Lambda in between --
// the passes of run_separable without the workspace.
static int run_small(const bdct_plan *p, Dir dir, const ExecGeom &g, cudaStream_t s)
{
    const int h = p->rows, w = p->cols;
    const Dir mdir = dir == DIR_SPEC ? DIR_RT : dir;  // the spectral direction uses the orthonormal pair
    const float *oph = p->ops + p->op_h_off[mdir];
    const float *opw = p->ops + p->op_w_off[mdir];
    const size_t per_dir = (size_t)h * h + (size_t)w * w;
    const bool pair = dir == DIR_RT || dir == DIR_SPEC;
    const int axis[4] = {0, 1, 1, 0};
    const float *ops[4] = {opw, oph, oph + per_dir, opw + per_dir};
    cudaError_t e = small_dense_run(h, w, pair ? 4 : 2, axis, ops, dir == DIR_SPEC ? p->spec_plain : nullptr, g, s);
    return e == cudaSuccess ? BDCT_OK : cuda_fail(e);
}

static int run_separable(const bdct_plan *p, Dir dir, const float *in, const long long *in_off, float *out,
                         const long long *out_off, long long count, cudaStream_t s)
{
    if (p->small) {
        ExecGeom g{in, out, count, 0, 0, 0, 0, in_off, out_off};
        return run_small(p, dir, g, s);
    }
    const int h = p->rows, w = p->cols;
    const long long hw = (long long)h * w;
    const Dir mdir = dir == DIR_SPEC ? DIR_RT : dir;  // the spectral direction uses the orthonormal pair
    const float *oph = p->ops + p->op_h_off[mdir];
    const float *opw = p->ops + p->op_w_off[mdir];
    const size_t per_dir = (size_t)h * h + (size_t)w * w;
    float *w1 = p->work;
    float *w2 = p->work + (size_t)p->chunk_arrays * hw;
    for (long long b0 = 0; b0 < count; b0 += p->chunk_arrays) {
        const long long nb = (count - b0) < p->chunk_arrays ? (count - b0) : p->chunk_arrays;
        const float *src = in + b0 * hw;
        float *dst = out + b0 * hw;
        const long long *ioff = in_off ? in_off + b0 : nullptr;
        const long long *ooff = out_off ? out_off + b0 : nullptr;
        cudaError_t e;
        // first pass: rows of the input into w1
        if (ioff) e = dense_pass_rows_indexed(in, ioff, w1, opw, h, w, nb, s);
        else e = dense_pass_rows(src, w1, opw, (int)(nb * h), w, s);
        if (dir != DIR_RT && dir != DIR_SPEC) {
            if (e == cudaSuccess) {
                if (ooff) e = dense_pass_cols_indexed(w1, out, ooff, oph, h, w, nb, s);
                else e = dense_pass_cols(w1, dst, oph, h, w, nb, s);
            }
        } else {
            // forward core, then the adjoint core (orthonormal pair)
            const float *ioph = oph + per_dir, *iopw = opw + per_dir;
            // the orthonormal spectrum of the chunk (times Lambda as it is
            // stored, for the spectral direction: Eq. 4)
            if (e == cudaSuccess)
                e = dense_pass_cols_lam(w1, w2, oph, h, w, nb, dir == DIR_SPEC ? p->spec_plain : nullptr, s);
            if (e == cudaSuccess) e = dense_pass_cols(w2, w1, ioph, h, w, nb, s);
            if (e == cudaSuccess) {
                if (ooff) e = dense_pass_rows_out_indexed(w1, out, ooff, iopw, h, w, nb, s);
                else e = dense_pass_rows(w1, dst, iopw, (int)(nb * h), w, s);
            }
        }
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return BDCT_OK;
}

// Orthonormal scales of one direction (the spectral composition of the
// kernel families without a fused spectral kernel runs the orthonormal forward
// and inverse around the diagonal, whatever the plan's normalization).
static DirScales ortho_scales(const bdct_plan *p, Dir dir)
{
    return DirScales{axis_scale(p->rows, dir, BDCT_NORM_ORTHO), axis_scale(p->cols, dir, BDCT_NORM_ORTHO)};
}

// One direction of a fused or tensor-core plan over geometry g (contiguous,
// indexed or tiled).  The spectral direction runs fused where a kernel has it
// (sides 8-32, tensor cores) and otherwise as orthonormal forward (in -> out),
// Lambda (in place), orthonormal inverse (out -> out, exact in place).
static int run_onchip(const bdct_plan *p, Dir dir, const ExecGeom &g0, cudaStream_t s)
{
    ExecGeom g = g0;
    cudaError_t e;
    if (p->variant == 3) {
        const Dir tdir = dir == DIR_SPEC ? DIR_RT : dir;  // tables: the orthonormal pair
        if (dir == DIR_SPEC) g.lam = p->spec_plain;
        e = tc_launch(p->rows, dir, p->tc_terms, g, p->tc_ops + p->tc_off[tdir], p->status, s);
        return e == cudaSuccess ? BDCT_OK : cuda_fail(e);
    }
    if (dir != DIR_SPEC) {
        e = fused_launch(p->rows, p->cols, dir, p->scales[dir], g, p->status, s);
        return e == cudaSuccess ? BDCT_OK : cuda_fail(e);
    }
    if (!ring_supported(p->rows, p->cols)) {
        g.lam = p->spec_fold;
        e = fused_launch(p->rows, p->cols, DIR_SPEC, p->scales[DIR_RT], g, p->status, s);
        return e == cudaSuccess ? BDCT_OK : cuda_fail(e);
    }
    if (p->rows == 64 && p->cols == 64) {
        // fused in the ring kernel: one read, one write
        g.lam = p->spec_fold;
        e = ring_launch(64, 64, DIR_SPEC, p->scales[DIR_RT], g, p->status, s);
        return e == cudaSuccess ? BDCT_OK : cuda_fail(e);
    }
    // the other ring shapes: the orthonormal forward multiplying its
    // coefficients by Lambda as it stores them, then the orthonormal inverse
    // in place
    g.lam = p->spec_plain;
    e = ring_forward_lam(p->rows, p->cols, ortho_scales(p, DIR_FWD), g, p->status, s);
    g.lam = nullptr;
    if (e == cudaSuccess) {
        ExecGeom gi = g;
        gi.in = g.out;
        gi.in_off = g.out_off;
        gi.ld_in = g.ld_out;
        e = fused_launch(p->rows, p->cols, DIR_INV, ortho_scales(p, DIR_INV), gi, p->status, s);
    }
    return e == cudaSuccess ? BDCT_OK : cuda_fail(e);
}

// Tensor-core separable passes (variant 4).  One direction of one slot over a
// chunk: rows of the input into the workspace (transposed), then the rows of
// that into the output (transposed back); lam (spectral) multiplies the
// spectrum in the second pass's epilogue.  The 8 x 8 Kronecker route is one
// pass per direction.
static cudaError_t tg_direction(const bdct_plan *p, int slot, const float *src, const long long *src_off, float *dst,
                                const long long *dst_off, long long nb, const float *lam, cudaStream_t s)
{
    const int h = p->rows, w = p->cols;
    if (p->tg_kron)
        return tg_pass(src, dst, src_off, dst_off, nb, 1, 64, p->tg_ops + p->tg_h[slot], p->tc_terms, lam, p->tg_abuf, p->status, s);
    cudaError_t e = tg_pass(src, p->work, src_off, nullptr, nb, h, w, p->tg_ops + p->tg_w[slot], p->tc_terms, nullptr,
                            p->tg_abuf, p->status, s);
    if (e == cudaSuccess)
        e = tg_pass(p->work, dst, nullptr, dst_off, nb, w, h, p->tg_ops + p->tg_h[slot], p->tc_terms, lam, p->tg_abuf, p->status, s);
    return e;
}

static int run_tg(const bdct_plan *p, Dir dir, const float *in, const long long *in_off, float *out,
                  const long long *out_off, long long count, cudaStream_t s)
{
    const long long hw = (long long)p->rows * p->cols;
    const bool inplace = (const void *)in == (const void *)out;
    for (long long b0 = 0; b0 < count; b0 += p->chunk_arrays) {
        const long long nb = (count - b0) < p->chunk_arrays ? (count - b0) : p->chunk_arrays;
        const float *src = in_off ? in : in + b0 * hw;
        float *dst = out_off ? out : out + b0 * hw;
        const long long *so = in_off ? in_off + b0 : nullptr;
        const long long *dof = out_off ? out_off + b0 : nullptr;
        cudaError_t e = cudaSuccess;
        if (dir == DIR_FWD || dir == DIR_INV) {
            const int slot = dir == DIR_FWD ? 0 : 1;
            if (p->tg_kron && inplace) {
                // one pass cannot run in place: through the workspace
                e = tg_pass(src, p->work, so, nullptr, nb, 1, 64, p->tg_ops + p->tg_h[slot], p->tc_terms, nullptr, p->tg_abuf,
                            p->status, s);
                ExecGeom g{p->work, dst, nb, 0, 0, 0, 0, nullptr, dof};
                if (e == cudaSuccess) e = copy_arrays(p->work, g, p->rows, p->cols, s);
            } else {
                e = tg_direction(p, slot, src, so, dst, dof, nb, nullptr, s);
            }
        } else {
            // round trip / spectral: orthonormal forward (times Lambda), then the inverse
            const float *lam = dir == DIR_SPEC ? p->spec_plain : nullptr;
            if (p->tg_kron) {
                e = tg_pass(src, p->work, so, nullptr, nb, 1, 64, p->tg_ops + p->tg_h[2], p->tc_terms, lam, p->tg_abuf, p->status, s);
                if (e == cudaSuccess)
                    e = tg_pass(p->work, dst, nullptr, dof, nb, 1, 64, p->tg_ops + p->tg_h[3], p->tc_terms, nullptr,
                                p->tg_abuf, p->status, s);
            } else {
                e = tg_direction(p, 2, src, so, dst, dof, nb, lam, s);
                if (e == cudaSuccess) e = tg_direction(p, 3, dst, dof, dst, dof, nb, nullptr, s);
            }
        }
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return BDCT_OK;
}

static int execute_dir(const bdct_plan *p, Dir dir, const float *in, const long long *in_off, float *out,
                       const long long *out_off, long long count, cudaStream_t s);

int bdct::plan_execute(const bdct_plan *p, Dir dir, const float *in, const long long *in_off, float *out,
                       const long long *out_off, long long count, cudaStream_t s)
{
    if (count <= 0) return BDCT_OK;
    if (dir == DIR_SPEC && !p->spec_plain) return BDCT_ERR_INVALID_ARG;  // no diagonal set
    if (!p->rp_bits) return execute_dir(p, dir, in, in_off, out, out_off, count, s);
    // range protection, per chunk of arrays: scale into the output, transform
    // in place there, scale back
    const long long hw = (long long)p->rows * p->cols;
    for (long long b0 = 0; b0 < count; b0 += p->rp_cap) {
        const long long nb = (count - b0) < p->rp_cap ? (count - b0) : p->rp_cap;
        const float *src = in_off ? in : in + b0 * hw;
        float *dst = out_off ? out : out + b0 * hw;
        const long long *so = in_off ? in_off + b0 : nullptr;
        const long long *dof = out_off ? out_off + b0 : nullptr;
        ExecGeom g{src, dst, nb, 0, 0, 0, 0, so, dof};
        cudaError_t e = range_prescale(g, p->rows, p->cols, p->rp_bits, s);
        if (e != cudaSuccess) return cuda_fail(e);
        const int st = execute_dir(p, dir, dst, dof, dst, dof, nb, s);
        if (st != BDCT_OK) return st;
        e = range_postscale(g, p->rows, p->cols, p->rp_bits, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return BDCT_OK;
}

static int execute_dir(const bdct_plan *p, Dir dir, const float *in, const long long *in_off, float *out,
                       const long long *out_off, long long count, cudaStream_t s)
{
    if (p->variant == 1 || p->variant == 3) {
        ExecGeom g{in, out, count, 0, 0, 0, 0, in_off, out_off};
        return run_onchip(p, dir, g, s);
    }
    if (p->variant == 4) return run_tg(p, dir, in, in_off, out, out_off, count, s);
    if (p->lines) {
        if (dir != DIR_SPEC) return run_lines(p, dir, p->scales[dir], in, in_off, out, out_off, count, s);
        // the orthonormal forward, its second pass storing the spectrum times
        // Lambda, then the orthonormal inverse in place
        int st = run_lines(p, DIR_FWD, ortho_scales(p, DIR_FWD), in, in_off, out, out_off, count, s, p->spec_plain);
        if (st == BDCT_OK) st = run_lines(p, DIR_INV, ortho_scales(p, DIR_INV), out, out_off, out, out_off, count, s);
        return st;
    }
    return run_separable(p, dir, in, in_off, out, out_off, count, s);
}

extern "C" int bdct_execute(const bdct_plan *plan, unsigned kind, const float *in, float *out,
                            size_t batch, void *stream)
{
    if (!plan) return BDCT_ERR_INVALID_ARG;
    Dir dir;
    int st = dir_of(kind, &dir);
    if (st != BDCT_OK) return st;
    if (!(plan->kind & kind)) return BDCT_ERR_KIND;
    if (batch == 0) return BDCT_OK;
    if (!in || !out) return BDCT_ERR_INVALID_ARG;
    if (((uintptr_t)in | (uintptr_t)out) & 15u) return BDCT_ERR_ALIGN;
    const size_t hw = (size_t)plan->rows * plan->cols;
    if (batch > (size_t)INT64_MAX / (hw * sizeof(float))) return BDCT_ERR_INVALID_ARG;
    if (ranges_partially_overlap(in, out, batch * hw * sizeof(float))) return BDCT_ERR_ALIAS;
    return plan_execute(plan, dir, in, nullptr, out, nullptr, (long long)batch, (cudaStream_t)stream);
}

extern "C" int bdct_forward(const bdct_plan *plan, const float *in, float *out, size_t batch, void *stream)
{
    return bdct_execute(plan, BDCT_FORWARD, in, out, batch, stream);
}

extern "C" int bdct_inverse(const bdct_plan *plan, const float *in, float *out, size_t batch, void *stream)
{
    return bdct_execute(plan, BDCT_INVERSE, in, out, batch, stream);
}

extern "C" int bdct_roundtrip(const bdct_plan *plan, const float *in, float *out, size_t batch, void *stream)
{
    return bdct_execute(plan, BDCT_ROUNDTRIP, in, out, batch, stream);
}

extern "C" int bdct_execute_tiled(const bdct_plan *plan, unsigned kind, const float *in, float *out,
                                  int img_rows, int img_cols, size_t ld_in, size_t ld_out, void *stream)
{
    if (!plan) return BDCT_ERR_INVALID_ARG;
    Dir dir;
    int st = dir_of(kind, &dir);
    if (st != BDCT_OK) return st;
    if (!(plan->kind & kind)) return BDCT_ERR_KIND;
    if (img_rows < 0 || img_cols < 0) return BDCT_ERR_INVALID_ARG;
    if (img_rows == 0 || img_cols == 0) return BDCT_OK;
    if (!in || !out) return BDCT_ERR_INVALID_ARG;
    if (img_rows % plan->rows || img_cols % plan->cols) return BDCT_ERR_UNSUPPORTED_SHAPE;
    if (ld_in < (size_t)img_cols || ld_out < (size_t)img_cols) return BDCT_ERR_INVALID_ARG;
    if ((((uintptr_t)in | (uintptr_t)out) & 15u) || (ld_in % 4) || (ld_out % 4)) return BDCT_ERR_ALIGN;
    if (plan->variant != 1 && plan->variant != 3 && !plan->small) return BDCT_ERR_PATH;
    const size_t span_in = ((size_t)(img_rows - 1) * ld_in + img_cols) * sizeof(float);
    const size_t span_out = ((size_t)(img_rows - 1) * ld_out + img_cols) * sizeof(float);
    if (in != out) {
        const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
        if (a < b + span_out && b < a + span_in) return BDCT_ERR_ALIAS;
    } else if (ld_in != ld_out) {
        return BDCT_ERR_ALIAS;
    }
    if (dir == DIR_SPEC && !plan->spec_plain) return BDCT_ERR_INVALID_ARG;  // no diagonal set
    const int tpr = img_cols / plan->cols;
    const long long tiles = (long long)(img_rows / plan->rows) * tpr;
    ExecGeom g{in, out, tiles, 1, tpr, (long long)ld_in, (long long)ld_out};
    auto run_tiles = [&](const ExecGeom &gg) {
        return plan->small ? run_small(plan, dir, gg, (cudaStream_t)stream)
                           : run_onchip(plan, dir, gg, (cudaStream_t)stream);
    };
    if (!plan->rp_bits) return run_tiles(g);
    // range protection: scale every block into the output, transform there in
    // place, scale back
    if (tiles > plan->rp_cap) return BDCT_ERR_UNSUPPORTED_SHAPE;
    cudaError_t e = range_prescale(g, plan->rows, plan->cols, plan->rp_bits, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    ExecGeom gi = g;
    gi.in = out;
    gi.ld_in = (long long)ld_out;
    st = run_tiles(gi);
    if (st != BDCT_OK) return st;
    e = range_postscale(g, plan->rows, plan->cols, plan->rp_bits, (cudaStream_t)stream);
    return e == cudaSuccess ? BDCT_OK : cuda_fail(e);
}

extern "C" int bdct_plan_set_range_protection(bdct_plan *plan, int on)
{
    if (!plan) return BDCT_ERR_INVALID_ARG;
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cur != plan->device && (e = cudaSetDevice(plan->device)) != cudaSuccess) return cuda_fail(e);
    int st = BDCT_OK;
    if (!on) {
        if (plan->rp_bits) {
            e = cudaDeviceSynchronize();
            cudaFree(plan->rp_bits);
            plan->rp_bits = nullptr;
            plan->rp_cap = 0;
            if (e != cudaSuccess) st = cuda_fail(e);
        }
    } else if (!plan->rp_bits) {
        const long long cap = 1ll << 20;  // arrays per chunk (4 MiB of exponent words)
        e = cudaMalloc(&plan->rp_bits, (size_t)cap * sizeof(unsigned int));
        if (e != cudaSuccess) {
            plan->rp_bits = nullptr;
            t_last_cuda_error = (int)e;
            st = BDCT_ERR_NO_MEMORY;
        } else {
            plan->rp_cap = cap;
        }
    }
    if (cur >= 0 && cur != plan->device) cudaSetDevice(cur);
    return st;
}

extern "C" int bdct_plan_set_spectral(bdct_plan *plan, const double *lambda)
{
    if (!plan || !lambda) return BDCT_ERR_INVALID_ARG;
    if (!(plan->kind & BDCT_SPECTRAL)) return BDCT_ERR_KIND;
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cur != plan->device) {
        e = cudaSetDevice(plan->device);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    const size_t n = (size_t)plan->rows * plan->cols;
    int st = BDCT_OK;
    double *d_lam = nullptr;
    if (!plan->spec_plain) {
        e = cudaMalloc(&plan->spec_plain, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&plan->spec_fold, n * sizeof(float));
        if (e != cudaSuccess) {
            if (plan->spec_plain) cudaFree(plan->spec_plain);
            plan->spec_plain = nullptr;
            t_last_cuda_error = (int)e;
            st = BDCT_ERR_NO_MEMORY;
        }
    }
    if (st == BDCT_OK) {
        e = cudaMalloc(&d_lam, n * sizeof(double));
        if (e != cudaSuccess) { t_last_cuda_error = (int)e; st = BDCT_ERR_NO_MEMORY; }
    }
    if (st == BDCT_OK) {
        e = cudaMemcpy(d_lam, lambda, n * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = spectral_gen_tables(d_lam, plan->spec_plain, plan->spec_fold, plan->rows, plan->cols, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e);
    }
    if (d_lam) cudaFree(d_lam);
    if (cur >= 0 && cur != plan->device) cudaSetDevice(cur);
    return st;
}

extern "C" int bdct_plan_get_info(const bdct_plan *plan, bdct_plan_info *info)
{
    if (!plan || !info) return BDCT_ERR_INVALID_ARG;
    info->rows = plan->rows;
    info->cols = plan->cols;
    info->kind = plan->kind;
    info->norm = plan->norm;
    info->path = plan->path;
    info->variant = plan->variant;
    info->workspace_bytes = plan->work_bytes;
    info->table_bytes = plan->table_bytes;
    return BDCT_OK;
}

extern "C" int bdct_plan_set_chunk_bytes(bdct_plan *plan, size_t bytes)
{
    if (!plan) return BDCT_ERR_INVALID_ARG;
    if ((plan->variant != 2 && plan->variant != 4) || plan->small) return BDCT_OK;
    const size_t arr_bytes = (size_t)plan->rows * plan->cols * sizeof(float);
    long long chunk = (long long)(bytes / arr_bytes);
    if (chunk < 1) chunk = 1;
    // the dense route keeps two buffers when it serves the round trip or the spectral direction
    const int nbuf = (plan->variant == 2 && !plan->lines && (plan->kind & (BDCT_ROUNDTRIP | BDCT_SPECTRAL))) ? 2 : 1;
    const size_t need = (size_t)chunk * arr_bytes * nbuf;
    if (need == plan->work_bytes) {
        plan->chunk_arrays = chunk;
        return BDCT_OK;
    }
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cur != plan->device && (e = cudaSetDevice(plan->device)) != cudaSuccess) return cuda_fail(e);
    float *w = nullptr;
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMalloc(&w, need);
    int st = BDCT_OK;
    if (e != cudaSuccess) {
        t_last_cuda_error = (int)e;
        st = BDCT_ERR_NO_MEMORY;
    } else {
        if (plan->work) cudaFree(plan->work);
        plan->work = w;
        plan->work_bytes = need;
        plan->chunk_arrays = chunk;
        if (plan->variant == 4 && (e = tg_alloc_split(plan)) != cudaSuccess) {
            t_last_cuda_error = (int)e;
            st = BDCT_ERR_NO_MEMORY;
        }
    }
    if (cur >= 0 && cur != plan->device) cudaSetDevice(cur);
    return st;
}

extern "C" int bdct_plan_device_status(const bdct_plan *plan, int clear)
{
    if (!plan) return BDCT_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e);
    unsigned int v = 0;
    e = cudaMemcpy(&v, plan->status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    if (clear && v) {
        e = cudaMemset(plan->status, 0, sizeof(v));
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return (int)v;
}

extern "C" const char *bdct_status_string(int status)
{
    switch (status) {
        case BDCT_OK: return "ok";
        case BDCT_ERR_INVALID_ARG: return "invalid argument";
        case BDCT_ERR_UNSUPPORTED_SHAPE: return "unsupported shape";
        case BDCT_ERR_KIND: return "direction not planned";
        case BDCT_ERR_ALIGN: return "misaligned pointer or stride";
        case BDCT_ERR_ALIAS: return "input and output overlap";
        case BDCT_ERR_CUDA: return "CUDA error";
        case BDCT_ERR_ARCH: return "device is not sm_103";
        case BDCT_ERR_DEVICE_TIMEOUT: return "device wait timed out";
        case BDCT_ERR_NO_MEMORY: return "device allocation failed";
        case BDCT_ERR_PATH: return "path unavailable for this shape";
        default: return "unknown status";
    }
}

extern "C" int bdct_last_cuda_error(void) { return t_last_cuda_error; }

extern "C" int bdct_version(void) { return 100; }
