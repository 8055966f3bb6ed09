// Host-buffer execution: copies in, transforms, copies out, overlapped.
//
// The paper measures complete calls including input copies (Sections 4.1,
// 4.2) and lists first-use and streaming workloads with data transfers as
// future work (Section 8).  These entry points take HOST buffers: the data
// moves in chunks through plan-owned device staging (four slots) so that
// the host-to-device copy of one chunk, the transforms of an earlier chunk
// and the device-to-host copy of one before it run at the same time on three
// streams (one per copy direction, one for the kernels).  A sequence of directions (for example forward
// then inverse) is applied to each chunk on the device, so intermediates never
// cross the host link.
#include <cuda_runtime.h>

#include <cstring>

#include "bdct_internal.h"
#include "plan.h"

using namespace bdct;

namespace {

int host_fail(cudaError_t e)
{
    (void)e;
    return BDCT_ERR_CUDA;
}

int dir_of_kind(unsigned k, Dir *d)
{
    switch (k) {
        case BDCT_FORWARD: *d = DIR_FWD; return BDCT_OK;
        case BDCT_INVERSE: *d = DIR_INV; return BDCT_OK;
        case BDCT_ROUNDTRIP: *d = DIR_RT; return BDCT_OK;
        case BDCT_SPECTRAL: *d = DIR_SPEC; return BDCT_OK;
        default: return BDCT_ERR_INVALID_ARG;
    }
}

}  // namespace

void bdct::host_staging_free(bdct_plan *p)
{
    for (int i = 0; i < kStageSlots; ++i) {
        for (int j = 0; j < 2; ++j)
            if (p->stage[i][j]) cudaFree(p->stage[i][j]);
        if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
        if (p->ev_done[i]) cudaEventDestroy(p->ev_done[i]);
        if (p->ev_out[i]) cudaEventDestroy(p->ev_out[i]);
    }
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->ev_end) cudaEventDestroy(p->ev_end);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->comp_stream) cudaStreamDestroy(p->comp_stream);
    if (p->d2h_stream) cudaStreamDestroy(p->d2h_stream);
    memset(p->stage, 0, sizeof(p->stage));
    memset(p->ev_in, 0, sizeof(p->ev_in));
    memset(p->ev_done, 0, sizeof(p->ev_done));
    memset(p->ev_out, 0, sizeof(p->ev_out));
    p->ev_start = p->ev_end = nullptr;
    p->copy_stream = p->comp_stream = p->d2h_stream = nullptr;
    p->stage_bytes = 0;
}

extern "C" int bdct_plan_set_host_staging(bdct_plan *plan, size_t chunk_bytes)
{
    if (!plan) return BDCT_ERR_INVALID_ARG;
    const size_t arr = (size_t)plan->rows * plan->cols * sizeof(float);
    if (chunk_bytes < arr) chunk_bytes = arr;
    chunk_bytes = (chunk_bytes / arr) * arr;
    host_staging_free(plan);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kStageSlots && e == cudaSuccess; ++i)
        for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaMalloc(&plan->stage[i][j], chunk_bytes);
    if (e != cudaSuccess) { host_staging_free(plan); return BDCT_ERR_NO_MEMORY; }
    for (int i = 0; i < kStageSlots && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&plan->ev_in[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_out[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_end, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->comp_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->d2h_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { host_staging_free(plan); return host_fail(e); }
    plan->stage_bytes = chunk_bytes;
    return BDCT_OK;
}

// Shared pipeline.  A chunk is `units` units of `unit_floats` floats at host
// offset unit * unit_floats; `run` applies the directions to a device chunk
// on the compute stream.  Host-to-device copies, transforms and
// device-to-host copies each have their own stream; events order them per
// chunk and keep a staging slot from being refilled before its previous
// contents were copied out.
template <typename RunFn>
static int pipeline(const bdct_plan *p, const float *h_in, float *h_out, long long nunits, size_t unit_floats,
                    long long units_per_chunk, cudaStream_t user, RunFn run)
{
    cudaError_t e = cudaEventRecord(p->ev_start, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_stream, p->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->comp_stream, p->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h_stream, p->ev_start, 0);
    if (e != cudaSuccess) return host_fail(e);
    const long long nch = (nunits + units_per_chunk - 1) / units_per_chunk;
    for (long long c = 0; c < nch; ++c) {
        const int slot = (int)(c % kStageSlots);
        const long long u0 = c * units_per_chunk;
        const long long nu = (nunits - u0) < units_per_chunk ? (nunits - u0) : units_per_chunk;
        const size_t bytes = (size_t)nu * unit_floats * sizeof(float);
        // copy in (after the slot's previous chunk has been copied out)
        if (c >= kStageSlots) e = cudaStreamWaitEvent(p->copy_stream, p->ev_out[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->stage[slot][0], h_in + (size_t)u0 * unit_floats, bytes, cudaMemcpyHostToDevice,
                                p->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_in[slot], p->copy_stream);
        // transform
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->comp_stream, p->ev_in[slot], 0);
        if (e != cudaSuccess) return host_fail(e);
        int which = 0;
        int st = run(p->stage[slot][0], p->stage[slot][1], nu, &which);
        if (st != BDCT_OK) return st;
        e = cudaEventRecord(p->ev_done[slot], p->comp_stream);
        // copy out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h_stream, p->ev_done[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out + (size_t)u0 * unit_floats, p->stage[slot][which], bytes,
                                cudaMemcpyDeviceToHost, p->d2h_stream);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_out[slot], p->d2h_stream);
        if (e != cudaSuccess) return host_fail(e);
    }
    // the caller's stream continues after the last copy out
    e = cudaEventRecord(p->ev_end, p->d2h_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, p->ev_end, 0);
    return e == cudaSuccess ? BDCT_OK : host_fail(e);
}

static int check_kinds(const bdct_plan *p, const unsigned *kinds, int nkinds, Dir *dirs)
{
    if (!kinds || nkinds < 1 || nkinds > 8) return BDCT_ERR_INVALID_ARG;
    for (int i = 0; i < nkinds; ++i) {
        int st = dir_of_kind(kinds[i], &dirs[i]);
        if (st != BDCT_OK) return st;
        if (!(p->kind & kinds[i])) return BDCT_ERR_KIND;
    }
    return BDCT_OK;
}

extern "C" int bdct_execute_host(const bdct_plan *plan, const unsigned *kinds, int nkinds, const float *h_in,
                                 float *h_out, size_t batch, void *stream)
{
    if (!plan) return BDCT_ERR_INVALID_ARG;
    Dir dirs[8];
    int st = check_kinds(plan, kinds, nkinds, dirs);
    if (st != BDCT_OK) return st;
    if (batch == 0) return BDCT_OK;
    if (!h_in || !h_out) return BDCT_ERR_INVALID_ARG;
    if (plan->stage_bytes == 0) return BDCT_ERR_INVALID_ARG;  // bdct_plan_set_host_staging first
    const size_t hw = (size_t)plan->rows * plan->cols;
    const long long per = (long long)(plan->stage_bytes / (hw * sizeof(float)));
    return pipeline(plan, h_in, h_out, (long long)batch, hw, per, (cudaStream_t)stream,
                    [&](float *a, float *b, long long n, int *which) {
                        float *src = a, *dst = b;
                        for (int i = 0; i < nkinds; ++i) {
                            int s2 = plan_execute(plan, dirs[i], src, nullptr, dst, nullptr, n, plan->comp_stream);
                            if (s2 != BDCT_OK) return s2;
                            float *t = src; src = dst; dst = t;
                        }
                        *which = (src == a) ? 0 : 1;
                        return (int)BDCT_OK;
                    });
}

extern "C" int bdct_execute_tiled_host(const bdct_plan *plan, const unsigned *kinds, int nkinds, const float *h_in,
                                       float *h_out, int img_rows, int img_cols, void *stream)
{
    if (!plan) return BDCT_ERR_INVALID_ARG;
    Dir dirs[8];
    int st = check_kinds(plan, kinds, nkinds, dirs);
    if (st != BDCT_OK) return st;
    if (img_rows < 0 || img_cols < 0) return BDCT_ERR_INVALID_ARG;
    if (img_rows == 0 || img_cols == 0) return BDCT_OK;
    if (!h_in || !h_out) return BDCT_ERR_INVALID_ARG;
    if (img_rows % plan->rows || img_cols % plan->cols || img_cols % 4) return BDCT_ERR_UNSUPPORTED_SHAPE;
    if (plan->stage_bytes == 0) return BDCT_ERR_INVALID_ARG;
    // a unit is one band of plan->rows image rows
    const size_t band = (size_t)plan->rows * img_cols;
    const long long per = (long long)(plan->stage_bytes / (band * sizeof(float)));
    if (per < 1) return BDCT_ERR_UNSUPPORTED_SHAPE;  // staging too small for one band
    return pipeline(plan, h_in, h_out, (long long)(img_rows / plan->rows), band, per, (cudaStream_t)stream,
                    [&](float *a, float *b, long long n, int *which) {
                        float *src = a, *dst = b;
                        for (int i = 0; i < nkinds; ++i) {
                            int s2 = bdct_execute_tiled(plan, kinds[i], src, dst, (int)(n * plan->rows), img_cols,
                                                        (size_t)img_cols, (size_t)img_cols, plan->comp_stream);
                            if (s2 != BDCT_OK) return s2;
                            float *t = src; src = dst; dst = t;
                        }
                        *which = (src == a) ? 0 : 1;
                        return (int)BDCT_OK;
                    });
}
