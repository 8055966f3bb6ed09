"""The allocation-free entry point against the FP64 oracle and the plan path.

bdct_execute_noalloc serves callers that cannot allocate device memory: it
needs no plan and keeps its scratch in a fixed device array.  These tests
call it through the C ABI several times in a row (different shapes and
directions, so each call reuses scratch an earlier one left behind; two of
the cases need more arrays than one chunk of the scratch holds) and compare
each result with the oracle -- the round trip with its exact result X -- and
with bdct_execute on the same input, within the parity tolerances of the
other GPU tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2609_28519_gb300 import inputs

pytestmark = pytest.mark.gpu


def _noalloc(L, rows, cols, kind, norm, x, y, stream):
    return L.bdct_execute_noalloc(rows, cols, kind, norm, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr()), x.numel() // (rows * cols),
                                  ctypes.c_void_p(stream))


def _check(o, got, ref, x, norm, kind_is_rt, tag):
    m = o.metrics(got, ref, x, output_relative=(norm == 1 and not kind_is_rt))
    assert m["nonfinite"] == 0, tag
    assert m["e_rel_max"] <= o.ERR_REL_TOL, (tag, m["e_rel_max"])
    assert m["max_abs_ratio_max"] <= o.MAX_ABS_TOL, (tag, m["max_abs_ratio_max"])


def test_noalloc_matches_oracle_and_plan_calls_in_a_row(oracle_mod, cuda_dev):
    import torch
    from paper_2609_28519_gb300 import Plan, native
    L = native.lib()
    stream = torch.cuda.current_stream(cuda_dev).cuda_stream
    # (rows, cols, kind, norm, batch); 512x512 round trips fit two arrays per
    # chunk of scratch and 256x256 forwards thirty, so those two run the chunk
    # loop (three and two chunks)
    cases = [(64, 64, native.FORWARD, 0, 37), (24, 40, native.ROUNDTRIP, 0, 5),
             (16, 16, native.INVERSE, 1, 200), (512, 512, native.ROUNDTRIP, 0, 5),
             (256, 256, native.FORWARD, 0, 40), (64, 64, native.FORWARD, 0, 37)]
    for (rows, cols, kind, norm, batch) in cases:
        x_np = inputs.uniform(900 + rows + cols + kind, batch, rows, cols)
        x = torch.from_numpy(x_np).to(cuda_dev)
        y = torch.full_like(x, float("nan"))
        assert _noalloc(L, rows, cols, kind, norm, x, y, stream) == 0
        ref_plan = Plan(rows, cols, kind=kind, norm=norm).execute(kind, x)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        rt = kind == native.ROUNDTRIP
        if kind == native.FORWARD:
            ref = oracle_mod.forward(x_np, norm)
        elif kind == native.INVERSE:
            ref = oracle_mod.inverse(x_np, norm)
        else:
            ref = x_np.astype(np.float64)
        tag = (rows, cols, kind, norm, batch)
        _check(oracle_mod, got, ref, x_np, norm, rt, ("oracle",) + tag)
        _check(oracle_mod, got, ref_plan.cpu().numpy().astype(np.float64), x_np, norm, rt, ("plan",) + tag)


def test_noalloc_rejects_oversize_and_bad_args(cuda_dev):
    import torch
    from paper_2609_28519_gb300 import native
    L = native.lib()
    x = torch.zeros(4, 16, 16, device=cuda_dev)
    vp = ctypes.c_void_p
    assert L.bdct_execute_noalloc(1024, 16, 1, 0, vp(x.data_ptr()), vp(x.data_ptr()), 1, None) == 2
    assert L.bdct_execute_noalloc(16, 513, 1, 0, vp(x.data_ptr()), vp(x.data_ptr()), 1, None) == 2
    assert L.bdct_execute_noalloc(16, 16, 3, 0, vp(x.data_ptr()), vp(x.data_ptr()), 1, None) == 1
    assert L.bdct_execute_noalloc(16, 16, 1, 0, None, None, 0, None) == 0
