"""The allocation-free entry point against the plan-based one.

bdct_execute_noalloc serves callers that cannot allocate device memory: it
needs no plan and keeps its scratch in a fixed device array.  These tests
call it through the C ABI twice in a row (different shapes and directions,
so the second call reuses scratch the first one left behind) and compare
each result with bdct_execute on the same input, within the parity
tolerances of the other GPU tests.  This file is collected last on purpose.
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


def test_noalloc_matches_plan_two_calls_in_a_row(oracle_mod, cuda_dev):
    import torch
    from paper_2609_28519_gb300 import Plan, native
    L = native.lib()
    stream = torch.cuda.current_stream(cuda_dev).cuda_stream
    cases = [(64, 64, native.FORWARD, 0, 37), (24, 40, native.ROUNDTRIP, 0, 5),
             (16, 16, native.INVERSE, 1, 200), (64, 64, native.FORWARD, 0, 37)]
    for (rows, cols, kind, norm, batch) in cases:
        x_np = inputs.uniform(900 + rows + cols + kind, batch, rows, cols)
        x = torch.from_numpy(x_np).to(cuda_dev)
        y = torch.full_like(x, float("nan"))
        assert _noalloc(L, rows, cols, kind, norm, x, y, stream) == 0
        ref = Plan(rows, cols, kind=kind, norm=norm).execute(kind, x)
        torch.cuda.synchronize()
        got, want = y.cpu().numpy(), ref.cpu().numpy()
        m = oracle_mod.metrics(got, want.astype(np.float64), x_np,
                               output_relative=(norm == 1 and kind != native.ROUNDTRIP))
        assert m["nonfinite"] == 0
        assert m["e_rel_max"] <= oracle_mod.ERR_REL_TOL, (rows, cols, kind, m["e_rel_max"])
        assert m["max_abs_ratio_max"] <= oracle_mod.MAX_ABS_TOL, (rows, cols, kind)


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
