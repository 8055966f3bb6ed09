// Internal definition of a plan (shared by the API and the ragged executor).
#pragma once

#include <cuda_bf16.h>

#include "bdct_internal.h"

// Staging slots of the host-buffer pipeline: with four, the copy-in of a
// chunk never waits for the copy-out of an earlier chunk in a short sequence.
constexpr int kStageSlots = 4;

struct bdct_plan {
    int rows = 0, cols = 0;
    unsigned kind = 0;
    int norm = 0;
    int path = 0;
    int variant = 0;  // 1 fused register tile, 2 separable passes, 3 tensor core, 4 tensor-core passes
    bool lines = false;  // separable passes through the FFT line engine (else dense GEMM passes)
    bool small = false;  // dense route on chip (both sides at most 64): no workspace
    float2 *line_tw = nullptr;        // line engine twiddles: w axis at 0, h axis at line_tw_h
    size_t line_tw_h = 0;
    int device = -1;
    bdct::DirScales scales[3];  // per Dir
    // separable route
    float *ops = nullptr;  // dense route: operator matrices, see op_h_off / op_w_off
    size_t op_h_off[3] = {0, 0, 0}, op_w_off[3] = {0, 0, 0};
    float *work = nullptr;
    size_t work_bytes = 0;
    long long chunk_arrays = 0;
    size_t table_bytes = 0;
    unsigned int *status = nullptr;  // device status word written by bounded waits
    // tensor-core route: per direction, the operator term tables
    __nv_bfloat16 *tc_ops = nullptr;
    size_t tc_off[3] = {0, 0, 0};
    int tc_terms = 3;
    // tensor-core separable passes (variant 4): blocked operator tables, per
    // slot (0 forward, 1 inverse in the plan's norm; 2 forward, 3 inverse
    // orthonormal, for the round trip and the spectral direction) and axis
    __nv_bfloat16 *tg_ops = nullptr;
    size_t tg_h[4] = {0, 0, 0, 0}, tg_w[4] = {0, 0, 0, 0};
    bool tg_kron = false;  // 8 x 8: one pass with the 64 x 64 Kronecker operator
    __nv_bfloat16 *tg_abuf = nullptr;  // input terms of the long-contraction kernel
    // spectral direction (bdct_plan_set_spectral): Lambda in FP32, and Lambda
    // folded with the squared scales for the unscaled fused cores (Prop. 1)
    float *spec_plain = nullptr, *spec_fold = nullptr;
    // range protection (bdct_plan_set_range_protection): one exponent word per
    // array of a chunk of at most rp_cap arrays; null = off
    unsigned int *rp_bits = nullptr;
    long long rp_cap = 0;
    // host-buffer execution (bdct_plan_set_host_staging): kStageSlots slots of
    // two device buffers, and streams/events of the copy-in / transform /
    // copy-out pipeline
    float *stage[kStageSlots][2] = {};
    size_t stage_bytes = 0;
    cudaStream_t copy_stream = nullptr, comp_stream = nullptr, d2h_stream = nullptr;
    cudaEvent_t ev_in[kStageSlots] = {}, ev_done[kStageSlots] = {}, ev_out[kStageSlots] = {};
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
};

namespace bdct {
// Release the host-staging buffers, streams and events of a plan.
void host_staging_free(bdct_plan *p);
// Run one direction of a plan on `count` arrays; with in_off/out_off (device
// arrays of element offsets) array b lives at in + in_off[b] and out +
// out_off[b], otherwise the batch is contiguous.  Returns a BDCT status.
int plan_execute(const bdct_plan *p, Dir dir, const float *in, const long long *in_off, float *out,
                 const long long *out_off, long long count, cudaStream_t s);
}  // namespace bdct
