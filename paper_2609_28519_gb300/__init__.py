"""Exact batched 2D DCT for GB300 (sm_103a).

Forward DCT-II, inverse DCT-III and the normalized round trip of Eq. 2 of the
BRiDCT paper, on batches of row-major float32 arrays, through the C ABI in
``include/bdct.h``.  ``native`` is the ctypes binding (no compute in Python),
``build`` compiles the CUDA library in-tree, ``inputs`` draws seeded
synthetic workloads.
"""
from .native import (  # noqa: F401
    FORWARD, INVERSE, ROUNDTRIP, NORM_ORTHO, NORM_NONE,
    PATH_AUTO, PATH_FP32, PATH_SPLIT_TC, PATH_SPLIT_HILO, PATH_BF16,
    BdctError, Plan, Ragged, lib,
)
